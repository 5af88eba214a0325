"""Property pins of the oracle over random sizes (hypothesis; skipped where it is absent).

Facts that hold for every size, checked on random n, PSF shapes (odd and even sides,
non-square), boundaries and data: the factored R(A) equals the explicit rearrangement of
the explicit blur (eq. (2.2)); a reflexive blur of a constant image returns that constant
(every output pixel sums the whole sum-1 PSF); kp_apply and kp_apply_t, Dx and Dx_t, Dy and
Dy_t are adjoint pairs; the rank of R(A) never exceeds min(s0, s1); the isotropic shrink
never lengthens a vector and keeps its direction.
"""
import numpy as np
import pytest

from oracle import kpsb_oracle as O

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

_SET = settings(max_examples=40, deadline=None, derandomize=True)


def _psf(seed, s0, s1):
    g = np.random.default_rng(seed)
    p = g.uniform(0.05, 1.0, size=(s0, s1))
    return p / p.sum()


@_SET
@given(n=st.integers(3, 9), s0=st.integers(1, 7), s1=st.integers(1, 7), bc=st.sampled_from([0, 1]),
       seed=st.integers(0, 2**31 - 1))
def test_factored_R_is_the_rearranged_blur(n, s0, s1, bc, seed):
    if bc == O.BC_REFLEXIVE and (s0 // 2 > n or s1 // 2 > n or s0 - 1 - s0 // 2 > n or s1 - 1 - s1 // 2 > n):
        return  # one reflection per side only
    psf = _psf(seed, s0, s1)
    R = O.rearrange(O.blur_matrix(psf, n, bc), n, n, n, n)
    F = O.r_factors(psf, n, bc)
    np.testing.assert_allclose(F.Kx @ (F.P.T @ F.Ky.T.toarray()), R, rtol=0, atol=1e-15)
    sv = np.linalg.svd(R, compute_uv=False)
    r = min(s0, s1)
    if r < len(sv):
        assert sv[r] <= 1e-12 * sv[0]


@_SET
@given(n=st.integers(3, 12), s=st.integers(1, 7), seed=st.integers(0, 2**31 - 1))
def test_reflexive_blur_of_a_constant_is_that_constant(n, s, seed):
    # with a half-sample mirror every output pixel sums all taps of a sum-1 PSF
    if s // 2 > n or s - 1 - s // 2 > n:
        return
    psf = _psf(seed, s, s)
    out = O.blur(psf, np.full((n, n), 2.5), O.BC_REFLEXIVE)
    np.testing.assert_allclose(out, 2.5, rtol=0, atol=1e-13)


@_SET
@given(n=st.integers(2, 10), k=st.integers(1, 4), seed=st.integers(0, 2**31 - 1))
def test_adjoint_pairs(n, k, seed):
    g = np.random.default_rng(seed)
    K = O.KPSum(Ax=g.standard_normal((k, n, n)), Ay=g.standard_normal((k, n, n)),
                sigma=g.uniform(0.1, 2.0, size=k))
    X, Y = g.standard_normal((n, n)), g.standard_normal((n, n))
    scale = np.abs(X).sum() * np.abs(Y).sum() * (1 + np.abs(K.Ax).max() * np.abs(K.Ay).max() * K.sigma.sum())
    assert abs(np.sum(O.kp_apply(K, X) * Y) - np.sum(X * O.kp_apply_t(K, Y))) <= 1e-12 * scale
    for D, Dt in ((O.Dx, O.Dx_t), (O.Dy, O.Dy_t)):
        assert abs(np.sum(D(X) * Y) - np.sum(X * Dt(Y))) <= 1e-12 * np.abs(X).sum() * np.abs(Y).sum()


@_SET
@given(cx=st.floats(-5, 5), cy=st.floats(-5, 5), v=st.floats(0, 3))
def test_isotropic_shrink_shortens_along_the_same_direction(cx, cy, v):
    dx, dy = O.shrink_iso(np.array(cx), np.array(cy), v)
    s, d = np.hypot(cx, cy), np.hypot(float(dx), float(dy))
    assert d <= s + 1e-12
    assert abs(d - max(s - v, 0.0)) <= 1e-12 * (1 + s)
    assert abs(float(dx) * cy - float(dy) * cx) <= 1e-12 * (1 + s * s)  # parallel to (cx, cy)
