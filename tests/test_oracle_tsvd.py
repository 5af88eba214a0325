"""Pins of the oracle's EGKB (Alg. 1), the nu_j rule, RSVD (Alg. 2) and Terms(A_k).

Independent facts used: LAPACK's full SVD of the explicit R(A); the closed-form singular
values from the s x s problem; the Golub-Kahan relations B Q = S C and B^T S = Q C^T;
orthonormality; and a bidiagonal test matrix whose GKB coefficients are known by hand.
"""
import math

import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I


def _ops(F):
    return (lambda v: O.r_apply(F, v)), (lambda u: O.r_apply_t(F, u))


@pytest.mark.parametrize("full", [True, False])
@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
def test_egkb_relations_and_orthogonality(full, bc):
    n = 16
    g = I.rng(40 + bc + 2 * full)
    psf = I.psf_gaussian_mixture(9, g)
    F = O.r_factors(psf, n, bc)
    B, BT = _ops(F)
    ts = O.egkb(B, BT, I.gaussian(n * n, g), k=4, p=3, full_reorth=full)
    C, S, Q = ts.info["C"], ts.info["S"], ts.info["Q"]
    kp = ts.kp
    assert kp == 7 and C.shape == (8, 7)
    bn = O.r_sigma_closed_form(F)[0]
    # B Q_kp = S_{kp+1} C  (Alg. 1 step 14)
    assert np.linalg.norm(B(Q) - S @ C) <= 1e-12 * bn
    # B^T S_kp = Q_kp C_kp^T  (upper part of C); the reorthogonalisation of q_j moves
    # it by the (growing) projections it removes, larger without reorthogonalising s_j
    assert np.linalg.norm(BT(S[:, :kp]) - Q @ C[:kp, :kp].T) <= (1e-12 if full else 1e-9) * bn
    assert np.linalg.norm(Q.T @ Q - np.eye(kp)) < 1e-13
    assert np.linalg.norm(S.T @ S - np.eye(kp + 1)) < (1e-13 if full else 1e-8)
    # lower bidiagonal with positive entries
    assert np.all(np.diag(C) > 0) and np.all(np.diag(C, -1) > 0)
    assert np.count_nonzero(np.triu(C, 1)) == 0 and np.count_nonzero(np.tril(C, -2)) == 0


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
def test_egkb_exact_when_space_exhausts_rank(bc):
    # rank(R(A)) <= s; with k_p >= rank the Ritz values equal the singular values
    n, s = 16, 5
    g = I.rng(50 + bc)
    psf = I.psf_random(s, g)
    F = O.r_factors(psf, n, bc)
    B, BT = _ops(F)
    R = O.rearrange(O.blur_matrix(psf, n, bc), n, n, n, n)
    sv = np.linalg.svd(R, compute_uv=False)
    ts = O.egkb(B, BT, I.gaussian(n * n, g), k=4, p=6)
    assert ts.info["breakdown"] is not None  # the Krylov space is exhausted at step s+1
    assert ts.kp == s
    np.testing.assert_allclose(ts.sigma, sv[:4], rtol=0, atol=1e-11 * sv[0])
    # Ritz vectors reproduce R(A)'s best rank-4 approximation
    Rk = ts.U @ np.diag(ts.sigma) @ ts.V.T
    np.testing.assert_allclose(np.linalg.norm(R - Rk), math.sqrt(np.sum(sv[4:] ** 2)),
                               rtol=1e-9, atol=1e-12)


def test_egkb_leading_values_vs_closed_form_large_n():
    # n = 64: no full SVD, the s x s closed form pins sigma_1..sigma_k
    pr = I.problem_small(0)
    n = 64
    F = O.r_factors(pr.psf, n, pr.bc)
    B, BT = _ops(F)
    cf = O.r_sigma_closed_form(F)
    g = I.rng(3)
    ts = O.egkb(B, BT, I.gaussian(n * n, g), k=5, p=4)
    np.testing.assert_allclose(ts.sigma, cf[:5], rtol=0, atol=1e-8 * cf[0])
    Ucf, scf, Vcf = O.r_tsvd_closed_form(F, 5)
    for i in range(3):  # well separated leading triplets: vectors up to sign
        assert abs(abs(ts.U[:, i] @ Ucf[:, i]) - 1) < 1e-8
        assert abs(abs(ts.V[:, i] @ Vcf[:, i]) - 1) < 1e-8


def _bidiag_problem(alpha, t):
    """Lower bidiagonal C (m x m-1 padded square) whose GKB from e_1 returns alpha, t."""
    m = len(alpha) + 1
    C = np.zeros((m, m))
    for i, a in enumerate(alpha):
        C[i, i] = a
        C[i + 1, i] = t[i]
    C[m - 1, m - 1] = 1e-3 * min(alpha)
    return C


def test_nu_rule_on_known_bidiagonal():
    # GKB of a lower bidiagonal matrix started at e_1 returns its own entries, so the
    # products zeta_j = alpha_j t_j and nu_j = sqrt(zeta_j zeta_{j-1}) are known in advance.
    alpha = [1.0, 0.9, 0.8, 0.5, 0.3, 0.9, 0.3, 0.2, 0.1, 0.05, 0.02, 0.01]
    t = [0.8, 0.7, 0.5, 0.3, 0.9, 0.4, 0.2, 0.1, 0.05, 0.02, 0.01, 0.005]
    C = _bidiag_problem(alpha, t)
    e1 = np.zeros(C.shape[0])
    e1[0] = 1.0
    B = lambda v: C @ v  # noqa: E731
    BT = lambda u: C.T @ u  # noqa: E731
    ts = O.egkb(B, BT, e1, k=10, p=2, tau=1e-6, full_reorth=True)
    np.testing.assert_allclose(ts.info["alpha"], alpha[:ts.kp], rtol=1e-14)
    np.testing.assert_allclose(ts.info["t"][1:], t[:ts.kp], rtol=1e-14)
    # zeta_j = alpha_j t_j (j >= 2 uses t_j = t[j-2]); by hand:
    zeta = {j: alpha[j - 1] * t[j - 2] for j in range(2, 10)}
    nu = {j: math.sqrt(zeta[j] * zeta[j - 1]) for j in range(3, 10)}
    # nu_3 > nu_4 > nu_5 < nu_6  ->  k = 5, then k_p = 7
    assert nu[3] > nu[4] > nu[5] < nu[6]
    assert ts.k == 5 and ts.kp == 7
    # relative tolerance branch: tau above nu_4/nu_3 stops at i = 4... but k >= 3 first
    ts2 = O.egkb(B, BT, e1, k=10, p=1, tau=nu[4] / nu[3] * 1.0001)
    assert ts2.k == 4 and ts2.kp == 5
    # cap: k never exceeds the given cap
    ts3 = O.egkb(B, BT, e1, k=3, p=2, tau=1e-12)
    assert ts3.k == 3 and ts3.kp == 5
    # the cap is taken as soon as i reaches it, also when the rule would fire one step later
    # (nu_6 > nu_5 would give k = 5 here)
    ts4 = O.egkb(B, BT, e1, k=4, p=2, tau=1e-12)
    assert ts4.k == 4 and ts4.kp == 6


def test_nu_rule_ignores_a_single_rise_of_zeta():
    # zeta_j = alpha_j t_j decays non-monotonically; the rule watches the two-term geometric
    # mean nu_j instead (Sec. 2.2).  Unit alpha and t_j = zeta_j: zeta rises at j = 4
    # (0.35 > 0.3) while nu_3 > nu_4 > nu_5 > nu_6 < nu_7, so k = 6, not 3.
    zeta = [0.5, 0.3, 0.35, 0.2, 0.1, 0.3, 0.05, 0.02, 0.01, 0.005, 0.002, 0.001]  # j = 2..13
    alpha = [1.0] * len(zeta)
    C = _bidiag_problem(alpha, zeta)
    e1 = np.zeros(C.shape[0])
    e1[0] = 1.0
    ts = O.egkb(lambda v: C @ v, lambda u: C.T @ u, e1, k=10, p=2, tau=1e-6)
    nu = {j: math.sqrt(zeta[j - 2] * zeta[j - 3]) for j in range(3, 9)}
    assert nu[3] > nu[4] > nu[5] > nu[6] < nu[7]
    assert ts.k == 6 and ts.kp == 8


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rsvd_is_rayleigh_ritz_on_the_power_range(q):
    # Alg. 2 with q power steps returns the Rayleigh-Ritz values of R(A) on
    # range((R R^T)^q R F): here k_p = 5 < rank 9, so the values depend on q
    n, s, k, kp = 10, 9, 3, 5
    g = I.rng(70 + q)
    psf = I.psf_random(s, g)
    F = O.r_factors(psf, n, O.BC_ZERO)
    B, BT = _ops(F)
    R = O.rearrange(O.blur_matrix(psf, n, O.BC_ZERO), n, n, n, n)
    Om = I.gaussian((n * n, kp), g)
    Y = R @ Om
    for _ in range(q):
        Y = R @ (R.T @ Y)
    Uy, sy, _ = np.linalg.svd(Y, full_matrices=False)  # orthonormal basis of range(Y)
    ref = np.linalg.svd(Uy.T @ R, compute_uv=False)[:k]
    ts = O.rsvd(B, BT, Om, k=k, q=q)
    np.testing.assert_allclose(ts.sigma, ref, rtol=0, atol=1e-9 * ref[0])
    if q < 2:  # each power step moves the values toward the true ones
        nxt = O.rsvd(B, BT, Om, k=k, q=q + 1).sigma
        sv = np.linalg.svd(R, compute_uv=False)[:k]
        assert np.abs(nxt - sv).max() < np.abs(ts.sigma - sv).max()


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
def test_rsvd_exact_when_oversampled_past_rank(bc):
    n, s = 16, 5
    g = I.rng(60 + bc)
    psf = I.psf_random(s, g)
    F = O.r_factors(psf, n, bc)
    B, BT = _ops(F)
    R = O.rearrange(O.blur_matrix(psf, n, bc), n, n, n, n)
    U, sv, Vt = np.linalg.svd(R)
    ts = O.rsvd(B, BT, I.gaussian((n * n, 8), g), k=4, q=1)
    np.testing.assert_allclose(ts.sigma, sv[:4], rtol=0, atol=1e-12 * sv[0])
    for i in range(4):
        assert abs(abs(ts.U[:, i] @ U[:, i]) - 1) < 1e-10
        assert abs(abs(ts.V[:, i] @ Vt[i]) - 1) < 1e-10


def test_rsvd_and_egkb_agree_on_smooth_psf():
    pr = I.problem_small(0)
    n = pr.n
    F = O.r_factors(pr.psf, n, pr.bc)
    B, BT = _ops(F)
    g = I.rng(8)
    cf = O.r_sigma_closed_form(F)
    te = O.egkb(B, BT, pr.start, k=5, p=3)
    tr = O.rsvd(B, BT, I.gaussian((n * n, 15), g), k=5)
    np.testing.assert_allclose(te.sigma, cf[:5], atol=1e-9 * cf[0])
    np.testing.assert_allclose(tr.sigma, cf[:5], atol=1e-9 * cf[0])


def test_kp_terms_reproduce_truncated_R():
    pr = I.problem_small(0)
    n = 16
    F = O.r_factors(pr.psf, n, pr.bc)
    B, BT = _ops(F)
    ts = O.egkb(B, BT, I.gaussian(n * n, I.rng(1)), k=3, p=6)
    K = O.kp_terms(ts, n)
    # R(sum sigma Ax (x) Ay) = sum sigma vec(Ax) vec(Ay)^T = U S V^T
    Rk = O.rearrange(O.kp_matrix(K), n, n, n, n)
    np.testing.assert_allclose(Rk, ts.U @ np.diag(ts.sigma) @ ts.V.T, atol=1e-13)
    for i in range(K.k):
        assert abs(np.linalg.norm(K.Ax[i]) - 1) < 1e-12 and abs(np.linalg.norm(K.Ay[i]) - 1) < 1e-12
        v = K.Ay[i].reshape(-1, order="F")  # vec order: ties go to the first entry of vec(Ay_i)
        assert v[np.argmax(np.abs(v))] > 0
