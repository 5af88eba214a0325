"""Pins of the oracle's shrinkage, CGLS (Alg. 5) and split Bregman (Alg. 3, 4).

Independent facts: brute-force minimisation of the scalar and 2-D shrinkage problems,
a dense least-squares solve of the augmented system, and a different convex solver
(Chambolle-Pock primal-dual, written here) for the TV-regularised objective on 8x8.
"""
import math

import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I


def test_shrink_is_scalar_argmin():
    lam, beta = 0.3, 0.02
    thr = O.sb_threshold(lam, beta)
    grid = np.linspace(-2, 2, 400001)
    for c in (-1.3, -0.12, -0.01, 0.0, 0.05, 0.1111, 0.9):
        f = lam**2 * (grid - c) ** 2 + beta * np.abs(grid)
        d_bf = grid[np.argmin(f)]
        assert abs(O.shrink(np.array(c), thr) - d_bf) <= 1e-5
    # the printed threshold 1/gamma = beta/lambda^2 is the argmin with 2*beta
    assert O.sb_threshold(lam, beta, "paper") == pytest.approx(O.sb_threshold(lam, 2 * beta))


def test_isotropic_shrink_is_2d_argmin():
    lam, beta = 0.5, 0.1
    thr = O.sb_threshold(lam, beta)
    g = np.linspace(-1, 1, 2001)
    X, Y = np.meshgrid(g, g, indexing="ij")
    for cx, cy in [(0.3, -0.2), (0.05, 0.04), (-0.6, 0.0), (0.0, 0.0), (0.1, 0.09)]:
        f = lam**2 * ((X - cx) ** 2 + (Y - cy) ** 2) + beta * np.sqrt(X**2 + Y**2)
        i = np.unravel_index(np.argmin(f), f.shape)
        dx, dy = O.shrink_iso(np.array(cx), np.array(cy), thr)
        assert abs(dx - X[i]) <= 1.5e-3 and abs(dy - Y[i]) <= 1.5e-3
    dx, dy = O.shrink_iso(np.zeros(3), np.zeros(3), thr)  # s = 0 gives d = 0
    assert np.all(dx == 0) and np.all(dy == 0)


def _small_problem(n=8, seed=123, eta=0.05):
    g = I.rng(seed)
    psf = I.psf_gaussian(5, 0.8, 1.2, 20.0)
    A = O.blur_matrix(psf, n, O.BC_ZERO)
    xt = I.image_piecewise_constant(n, g)
    b = O.array(A @ O.vec(xt), n, n)
    b = b + I.noise_vector(b, eta, I.gaussian((n, n), g))
    Af = lambda X: O.array(A @ O.vec(X), n, n)  # noqa: E731
    ATf = lambda Y: O.array(A.T @ O.vec(Y), n, n)  # noqa: E731
    return A, Af, ATf, b, xt


def test_cgls_solves_augmented_least_squares():
    n = 8
    A, Af, ATf, b, _ = _small_problem(n)
    g = I.rng(5)
    mu, lam = 0.7, 0.3
    hx, hy = g.standard_normal((n, n)), g.standard_normal((n, n))
    L = O.L_matrix(n)
    Ah = np.vstack([math.sqrt(mu) * A, lam * np.kron(L, np.eye(n)), lam * np.kron(np.eye(n), L)])
    bh = np.concatenate([math.sqrt(mu) * O.vec(b), lam * O.vec(hx), lam * O.vec(hy)])
    x_ls = np.linalg.lstsq(Ah, bh, rcond=None)[0]

    def Ahat(X):
        return (math.sqrt(mu) * Af(X), lam * O.Dx(X), lam * O.Dy(X))

    def AhatT(r):
        return math.sqrt(mu) * ATf(r[0]) + lam * O.Dx_t(r[1]) + lam * O.Dy_t(r[2])

    res = O.cgls(Ahat, AhatT, (math.sqrt(mu) * b, lam * hx, lam * hy), (n, n), i_max=500, tau=1e-15)
    np.testing.assert_allclose(O.vec(res.x), x_ls, rtol=0, atol=1e-10 * np.abs(x_ls).max())
    # the relative-change stop of (5.1) ends earlier and the iteration count is reported
    res2 = O.cgls(Ahat, AhatT, (math.sqrt(mu) * b, lam * hx, lam * hy), (n, n), i_max=500, tau=1e-4)
    assert res2.iters < res.iters and res2.rc < 1e-4
    res3 = O.cgls(Ahat, AhatT, (math.sqrt(mu) * b, lam * hx, lam * hy), (n, n), i_max=7, fixed=True)
    assert res3.iters == 7


@pytest.mark.parametrize("i", [1, 3, 6])
def test_cgls_iterate_minimises_over_the_krylov_space(i):
    # the i-th CGLS iterate from x = 0 is argmin ||Ahat x - bhat|| over the Krylov space
    # K_i(Ahat^T Ahat, Ahat^T bhat) (textbook property of CG on the normal equations); the
    # reference solves that i-dimensional least-squares problem in an orthonormal basis
    n = 8
    A, Af, ATf, b, _ = _small_problem(n)
    mu, lam = 0.7, 0.3
    g = I.rng(12)
    hx, hy = g.standard_normal((n, n)), g.standard_normal((n, n))
    L = O.L_matrix(n)
    Ah = np.vstack([math.sqrt(mu) * A, lam * np.kron(L, np.eye(n)), lam * np.kron(np.eye(n), L)])
    bh = np.concatenate([math.sqrt(mu) * O.vec(b), lam * O.vec(hx), lam * O.vec(hy)])
    G = Ah.T @ Ah
    basis = []
    v = Ah.T @ bh
    for _ in range(i):  # Lanczos-style orthonormal basis with full reorthogonalisation
        for q in basis:
            v = v - (q @ v) * q
        for q in basis:
            v = v - (q @ v) * q
        basis.append(v / np.linalg.norm(v))
        v = G @ basis[-1]
    Qk = np.stack(basis, axis=1)
    x_ref = Qk @ np.linalg.lstsq(Ah @ Qk, bh, rcond=None)[0]

    def Ahat(X):
        return (math.sqrt(mu) * Af(X), lam * O.Dx(X), lam * O.Dy(X))

    def AhatT(r):
        return math.sqrt(mu) * ATf(r[0]) + lam * O.Dx_t(r[1]) + lam * O.Dy_t(r[2])

    res = O.cgls(Ahat, AhatT, (math.sqrt(mu) * b, lam * hx, lam * hy), (n, n), i_max=i, fixed=True)
    np.testing.assert_allclose(O.vec(res.x), x_ref, rtol=0, atol=1e-10 * np.abs(x_ref).max())


def _chambolle_pock(A, b, mu, beta, iso, iters):
    """Primal-dual solve of min mu||Ax-b||^2 + beta TV(x) (a different algorithm)."""
    n = b.shape[0]
    N = n * n
    L = O.L_matrix(n)
    D = np.vstack([np.kron(L, np.eye(n)), np.kron(np.eye(n), L)])
    step = 0.99 / np.linalg.norm(D, 2)
    M = np.linalg.inv(np.eye(N) + 2 * step * mu * A.T @ A)
    rhs0 = 2 * step * mu * A.T @ O.vec(b)
    x = np.zeros(N)
    xb = x.copy()
    y = np.zeros(2 * N)
    for _ in range(iters):
        y = y + step * (D @ xb)
        if iso:
            yy = y.reshape(2, N)
            y = (yy / np.maximum(1.0, np.hypot(yy[0], yy[1]) / beta)).reshape(-1)
        else:
            y = np.clip(y, -beta, beta)
        xn = M @ (x - step * (D.T @ y) + rhs0)
        xb = 2 * xn - x
        x = xn
    return O.array(x, n, n)


@pytest.mark.parametrize("iso,mu", [(False, 1.0), (True, 1.0), (False, 0.4), (True, 2.5)])
def test_split_bregman_reaches_tv_minimiser(iso, mu):
    # mu != 1 separates the minimisers (they move by ~0.1 between mu = 1 and 0.4 or 2.5 here),
    # so a sqrt(mu) dropped from the operator or the data block of A-hat fails
    n = 8
    A, Af, ATf, b, _ = _small_problem(n)
    lam, beta = 0.3, 0.01
    x_cp = _chambolle_pock(A, b, mu, beta, iso, 60000)
    res = O.split_bregman(Af, ATf, b, mu, lam, beta, iso, iters=1500, tau_cgls=1e-15, i_max=400)
    tol = 1e-4 if iso else 1e-10  # isotropic SB converges more slowly
    assert np.abs(res.x - x_cp).max() < tol
    if mu != 1.0:
        assert np.abs(_chambolle_pock(A, b, 1.0, beta, iso, 60000) - x_cp).max() > 1e-2
    # the printed threshold 1/gamma solves the problem with 2*beta instead
    res_p = O.split_bregman(Af, ATf, b, mu, lam, beta, iso, iters=300, tau_cgls=1e-15, i_max=400,
                            threshold_rule="paper")
    assert np.abs(res_p.x - x_cp).max() > 1e-2


def test_split_bregman_stopping_and_counts():
    n = 8
    A, Af, ATf, b, xt = _small_problem(n)
    res = O.split_bregman(Af, ATf, b, 1.0, 0.3, 0.01, False, iters=50, tau_sb=1e-3, x_true=xt)
    assert res.l_end < 50 and res.rc_sb < 1e-3
    assert res.iota_total == sum(h["iters"] for h in res.history)
    res2 = O.split_bregman(Af, ATf, b, 1.0, 0.3, 0.01, False, iters=4, i_max=6, fixed_inner=True)
    assert res2.l_end == 4 and res2.iota_total == 24
    # deblurring improves on the data (positive ISNR) for this well-posed toy case
    assert O.isnr(res.x, b, xt) > 0


def test_relative_changes_are_the_steps_between_iterates():
    # RC_CGLS (5.1) is the relative change of the CGLS iterate and RC_SB (5.2) that of the
    # outer iterate against the previous one, from x^(0) = b (Alg. 3/4 initialisation):
    # both checked against the differences of consecutive iterates
    n = 8
    A, Af, ATf, b, _ = _small_problem(n)
    mu, lam = 0.7, 0.3
    g = I.rng(9)
    hx, hy = g.standard_normal((n, n)), g.standard_normal((n, n))

    def Ahat(X):
        return (math.sqrt(mu) * Af(X), lam * O.Dx(X), lam * O.Dy(X))

    def AhatT(r):
        return math.sqrt(mu) * ATf(r[0]) + lam * O.Dx_t(r[1]) + lam * O.Dy_t(r[2])

    bh = (math.sqrt(mu) * b, lam * hx, lam * hy)
    xs = [O.cgls(Ahat, AhatT, bh, (n, n), i_max=i, fixed=True) for i in (1, 5, 6)]
    assert xs[0].rc == pytest.approx(1.0, rel=1e-12)  # from x^(0) = 0 the first step is all change
    step = np.linalg.norm(xs[2].x - xs[1].x) / np.linalg.norm(xs[2].x)
    assert xs[2].rc == pytest.approx(step, rel=1e-9)
    # the tolerance stop ends at the first iteration whose change is below tau
    rcs = [O.cgls(Ahat, AhatT, bh, (n, n), i_max=i, fixed=True).rc for i in range(1, 7)]
    tau = rcs[5] * (1 + 1e-9)
    first = next(i for i, r in enumerate(rcs, start=1) if r < tau)
    assert O.cgls(Ahat, AhatT, bh, (n, n), i_max=50, tau=tau).iters == first

    sb = [O.split_bregman(Af, ATf, b, 1.0, 0.3, 0.01, False, iters=i, i_max=30, fixed_inner=True)
          for i in (1, 2)]
    assert sb[0].rc_sb == pytest.approx(np.linalg.norm(sb[0].x - b) / np.linalg.norm(b), rel=1e-12)
    assert sb[1].rc_sb == pytest.approx(
        np.linalg.norm(sb[1].x - sb[0].x) / np.linalg.norm(sb[0].x), rel=1e-9)
    assert [h["rc_sb"] for h in sb[1].history][0] == pytest.approx(sb[0].rc_sb, rel=1e-12)

