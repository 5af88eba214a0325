"""Pins of the oracle's blur operator, rearrangement R(A), index maps and KP identities.

Each check compares the oracle with something other than itself: SciPy's 2-D
convolution, the Kronecker-product rearrangement identity on random matrices, LAPACK's
full SVD of the explicit R(A), brute-force sums, or the explicit Kronecker matrix.
"""
import numpy as np
import pytest
from scipy.signal import convolve2d

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
@pytest.mark.parametrize("n,s", [(8, 5), (9, 3), (12, 7), (6, 6)])
def test_blur_matches_scipy_convolution(bc, n, s):
    g = I.rng(11 + n + s + bc)
    psf = I.psf_random(s, g)
    X = g.uniform(size=(n, n))
    A = O.blur_matrix(psf, n, bc)
    got = O.array(A @ O.vec(X), n, n)
    if s % 2 == 1:
        ref = convolve2d(X, psf, mode="same", boundary="fill" if bc == O.BC_ZERO else "symm")
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)
    # the vectorised tap sum equals the explicit matrix (same arithmetic, other order)
    np.testing.assert_allclose(O.blur(psf, X, bc), got, rtol=0, atol=1e-14)


def test_reflexive_is_half_sample_mirror():
    # a delta PSF shifted by one pixel copies x[0] into the first output row (x[-1] = x[0])
    psf = np.zeros((3, 3))
    psf[2, 1] = 1.0  # tap a = 2: output row r reads input row r - 2 + 1 = r - 1
    X = np.arange(16.0).reshape(4, 4)
    B = O.blur(psf, X, O.BC_REFLEXIVE)
    np.testing.assert_array_equal(B[0], X[0])
    np.testing.assert_array_equal(B[1:], X[:-1])
    Bz = O.blur(psf, X, O.BC_ZERO)
    np.testing.assert_array_equal(Bz[0], 0.0)


def test_reflexive_extension_bounds():
    # one half-sample reflection per side: -n..-1 -> n-1..0 and n..2n-1 -> n-1..0; a PSF
    # reaching further than the image is refused
    n = 5
    assert [O.ext(q, n, O.BC_REFLEXIVE) for q in range(-n, 0)] == list(range(n - 1, -1, -1))
    assert [O.ext(q, n, O.BC_REFLEXIVE) for q in range(n, 2 * n)] == list(range(n - 1, -1, -1))
    assert [O.ext(q, n, O.BC_ZERO) for q in (-1, n)] == [None, None]
    for q in (-n - 1, 2 * n):
        with pytest.raises(ValueError):
            O.ext(q, n, O.BC_REFLEXIVE)


def test_rearrangement_of_kronecker_product():
    # R(B (x) C) = vec(B) vec(C)^T (the identity behind Theorem 2.1)
    g = I.rng(5)
    for (m1, n1, m2, n2) in [(3, 4, 2, 5), (4, 4, 4, 4), (1, 3, 2, 1)]:
        Bm = g.standard_normal((m1, n1))
        Cm = g.standard_normal((m2, n2))
        R = O.rearrange(np.kron(Bm, Cm), m1, n1, m2, n2)
        np.testing.assert_array_equal(R, np.outer(O.vec(Bm), O.vec(Cm)))


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
@pytest.mark.parametrize("n,s", [(8, 5), (10, 9), (7, 7), (8, 4)])
def test_factored_R_equals_explicit_rearrangement(bc, n, s):
    g = I.rng(100 + 3 * n + s + bc)
    psf = I.psf_random(s, g)
    R = O.rearrange(O.blur_matrix(psf, n, bc), n, n, n, n)
    F = O.r_factors(psf, n, bc)
    dense = (F.Kx @ (F.P.T @ F.Ky.T.toarray()))
    np.testing.assert_allclose(dense, R, rtol=0, atol=1e-15)
    V = g.standard_normal((n * n, 3))
    np.testing.assert_allclose(O.r_apply(F, V), R @ V, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(O.r_apply_t(F, V), R.T @ V, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
@pytest.mark.parametrize("shape", [(3, 7), (7, 3), (5, 1)])
def test_non_square_psf(bc, shape):
    # s0 != s1 separates the row (y) factor from the column (x) factor: the blur against
    # scipy's 2-D convolution, and R(A) from its factors against the explicit rearrangement
    n = 9
    g = I.rng(300 + 10 * shape[0] + shape[1] + bc)
    psf = g.uniform(0.05, 1.0, size=shape)
    psf /= psf.sum()
    X = g.uniform(size=(n, n))
    A = O.blur_matrix(psf, n, bc)
    ref = convolve2d(X, psf, mode="same", boundary="fill" if bc == O.BC_ZERO else "symm")
    np.testing.assert_allclose(O.array(A @ O.vec(X), n, n), ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose(O.blur(psf, X, bc), ref, rtol=0, atol=1e-14)
    R = O.rearrange(A, n, n, n, n)
    F = O.r_factors(psf, n, bc)
    np.testing.assert_allclose(F.Kx @ (F.P.T @ F.Ky.T.toarray()), R, rtol=0, atol=1e-15)
    V = g.standard_normal((n * n, 2))
    np.testing.assert_allclose(O.r_apply(F, V), R @ V, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(O.r_apply_t(F, V), R.T @ V, rtol=1e-13, atol=1e-14)
    sv = np.linalg.svd(R, compute_uv=False)
    r = min(shape)
    np.testing.assert_allclose(O.r_sigma_closed_form(F)[:r], sv[:r], rtol=0, atol=1e-12 * sv[0])
    assert sv[r] < 1e-12 * sv[0]  # rank <= min(s0, s1)


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
def test_index_maps_gather_is_bit_exact(bc):
    n, s = 8, 5
    g = I.rng(7 + bc)
    psf = I.psf_random(s, g)
    R = O.rearrange(O.blur_matrix(psf, n, bc), n, n, n, n)
    row_map, col_map = O.r_index_maps(psf.shape, n, bc)
    G = np.zeros_like(R)
    for ri, bs in enumerate(row_map):
        for ci, as_ in enumerate(col_map):
            acc = 0.0
            for b in bs:
                for a in as_:
                    acc += psf[a, b]
            G[ri, ci] = acc
    # entries with one contribution are copies; reflexive corners sum <= 4 taps
    np.testing.assert_allclose(G, R, rtol=0, atol=1e-16)
    nnz = [len(b) for b in row_map]
    assert max(nnz) <= (1 if bc == O.BC_ZERO else 3)


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
@pytest.mark.parametrize("n,s", [(8, 5), (12, 9), (16, 7), (10, 10)])
def test_closed_form_singular_values_match_lapack(bc, n, s):
    g = I.rng(200 + n + s + bc)
    psf = I.psf_random(s, g)
    R = O.rearrange(O.blur_matrix(psf, n, bc), n, n, n, n)
    sv = np.linalg.svd(R, compute_uv=False)
    cf = O.r_sigma_closed_form(O.r_factors(psf, n, bc))
    assert np.all(sv[len(cf):] <= 1e-12 * sv[0])  # rank(R(A)) <= s
    np.testing.assert_allclose(cf, sv[:len(cf)], rtol=0, atol=1e-12 * sv[0])


def test_separable_psf_gives_rank_one():
    g = I.rng(9)
    psf = I.psf_separable(5, g)
    for bc in (O.BC_ZERO, O.BC_REFLEXIVE):
        R = O.rearrange(O.blur_matrix(psf, 8, bc), 8, 8, 8, 8)
        sv = np.linalg.svd(R, compute_uv=False)
        assert sv[1] < 1e-14 * sv[0]
        cf = O.r_sigma_closed_form(O.r_factors(psf, 8, bc))
        assert cf[1] < 1e-13 * cf[0]


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
def test_van_loan_pitsianis_identity(bc):
    # ||A - sum_{i<=r} sigma_i Ax_i (x) Ay_i||_F^2 = sum_{i>r} sigma_i^2   (Theorem 2.1)
    n = 6
    g = I.rng(31 + bc)
    psf = I.psf_random(5, g)
    A = O.blur_matrix(psf, n, bc)
    R = O.rearrange(A, n, n, n, n)
    U, sv, Vt = np.linalg.svd(R)
    for r in (1, 2, 4, 5):
        ts = O.TSVD(U=U[:, :r], sigma=sv[:r], V=Vt[:r].T, k=r, kp=r)
        K = O.kp_terms(ts, n)
        err2 = np.linalg.norm(A - O.kp_matrix(K)) ** 2
        np.testing.assert_allclose(err2, np.sum(sv[r:] ** 2), rtol=1e-10, atol=1e-24)
    ts = O.TSVD(U=U[:, :5], sigma=sv[:5], V=Vt[:5].T, k=5, kp=5)
    np.testing.assert_allclose(O.kp_matrix(O.kp_terms(ts, n)), A, atol=1e-13)


def test_kp_apply_is_kronecker_matvec_and_adjoint():
    # (Ax (x) Ay) vec(X) = vec(Ay X Ax^T)  (Sec. 4.2); transpose is the adjoint
    g = I.rng(77)
    n, k = 7, 3
    K = O.KPSum(Ax=g.standard_normal((k, n, n)), Ay=g.standard_normal((k, n, n)),
                sigma=g.uniform(0.5, 2.0, size=k))
    M = O.kp_matrix(K)
    X = g.standard_normal((n, n))
    Y = g.standard_normal((n, n))
    np.testing.assert_allclose(O.vec(O.kp_apply(K, X)), M @ O.vec(X), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.vec(O.kp_apply_t(K, Y)), M.T @ O.vec(Y), rtol=1e-13, atol=1e-13)


def test_difference_operators_match_kronecker_forms():
    n = 6
    L = O.L_matrix(n)
    assert np.all(L[-1] == 0) and L[0, 0] == 0.5 and L[0, 1] == -0.5
    g = I.rng(3)
    X = g.standard_normal((n, n))
    I_n = np.eye(n)
    np.testing.assert_allclose(O.vec(O.Dx(X)), np.kron(L, I_n) @ O.vec(X), atol=1e-15)
    np.testing.assert_allclose(O.vec(O.Dy(X)), np.kron(I_n, L) @ O.vec(X), atol=1e-15)
    Y = g.standard_normal((n, n))
    np.testing.assert_allclose(O.vec(O.Dx_t(Y)), np.kron(L, I_n).T @ O.vec(Y), atol=1e-15)
    np.testing.assert_allclose(O.vec(O.Dy_t(Y)), np.kron(I_n, L).T @ O.vec(Y), atol=1e-15)


def test_metrics_special_cases():
    g = I.rng(4)
    xt = g.uniform(size=(5, 5))
    b = xt + 0.1 * g.standard_normal((5, 5))
    assert O.rel_error(xt, xt) == 0.0
    assert O.rel_error(3 * xt, xt) == pytest.approx(2.0, rel=1e-14)  # error measured in ||x_true||
    assert O.rel_error(np.zeros_like(xt), xt) == pytest.approx(1.0, rel=1e-14)
    assert abs(O.isnr(b, b, xt)) < 1e-12  # x = b: no improvement
    x_half = xt + 0.5 * (b - xt)  # error halved: +6.02 dB
    np.testing.assert_allclose(O.isnr(x_half, b, xt), 20 * np.log10(2.0), rtol=1e-12)
    eta = 0.05
    zeta = g.standard_normal((5, 5))
    noisy = xt + I.noise_vector(xt, eta, zeta)
    np.testing.assert_allclose(O.snr(xt, noisy), -20 * np.log10(eta), rtol=1e-12)
