"""The one-block EGKB (single precision, n <= 128): one thread block runs the whole recurrence
of Alg. 1 (R(A) through the index map of eq. (2.2), CGS2 reorthogonalisation, the nu rule of
eq. (2.6), breakdowns), the FP64 SVD of the bidiagonal C (step 15) and the Ritz vectors and terms
(steps 16-17, Theorem 2.1); every problem of a batch shares the same two launches.

Bounds as for the multi-kernel path (tests/test_gpu_kpbuild.py): leading sigma within
1e-4 sigma_1 of the oracle's Alg. 1 on the same start vector and of the closed form,
well-separated leading factor pairs equal up to sign (|<u, u_ref>| within 1e-3 of 1).  Against
the multi-kernel path (KPSB_EGKB_BLOCK=0) on the same inputs: the same rank and sigma within
2e-5 sigma_1 (both are FP32 bases with FP64 scalars; they differ in summation order only).
A problem alone and in a batch: identical bits.
"""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _vecs(K, kp):
    Ax, Ay, sig = K.kp_get_factors(kp)
    U = np.stack([O.vec(a) for a in Ax], axis=1).astype(np.float64)
    V = np.stack([O.vec(a) for a in Ay], axis=1).astype(np.float64)
    return U, sig, V


def _psf(seed, s=31):
    return I.psf_gaussian_mixture(s, I.rng(seed))


@pytest.mark.parametrize("one_sided", [False, True])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n", [40, 100, 128])
def test_block_egkb_matches_oracle(n, bc, one_sided):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    psf = _psf(300 + n + bc)
    start = I.gaussian(n * n, I.rng(7 + n)).astype(np.float32)
    tau, p = 1e-3, 8
    kp = K.kp_build(psf, n, bc, tau, K.EGKB, p=p, start=start, one_sided=one_sided)
    inf = K.kp_info(kp)
    F = O.r_factors(psf, n, bc)
    ref = O.egkb(lambda v: O.r_apply(F, v), lambda u: O.r_apply_t(F, u), start.astype(np.float64), 30, p,
                 tau=tau, full_reorth=not one_sided)
    if inf["k"] != ref.k:  # the rule may flip only where nu is flat at the deciding index
        j = min(inf["k"], ref.k) + 1
        nu = ref.info["nu"]
        assert abs(nu[j] - nu[j - 1]) < 1e-4 * nu[j - 1]
    k = min(inf["k"], ref.k)
    U, sig, V = _vecs(K, kp)
    cf = O.r_sigma_closed_form(F)
    np.testing.assert_allclose(sig[:k], ref.sigma[:k], rtol=0, atol=1e-4 * ref.sigma[0])
    np.testing.assert_allclose(sig[:k], cf[:k], rtol=0, atol=1e-4 * cf[0])
    for i in range(min(k, 4)):
        gap = min(abs(ref.sigma[i] - ref.sigma[i + 1]), abs(ref.sigma[i - 1] - ref.sigma[i]) if i else np.inf)
        if gap < 1e-2 * ref.sigma[0]:
            continue
        assert abs(abs(U[:, i] @ ref.U[:, i]) - 1) < 1e-3
        assert abs(abs(V[:, i] @ ref.V[:, i]) - 1) < 1e-3
    Ax, Ay, _ = K.kp_get_factors(kp)
    for i in range(inf["k"]):  # unit factors, sign convention in vec order
        assert abs(np.linalg.norm(Ax[i]) - 1) < 1e-5 and abs(np.linalg.norm(Ay[i]) - 1) < 1e-5
        v = Ay[i].reshape(-1, order="F")
        assert v[np.argmax(np.abs(v))] > 0


@pytest.mark.parametrize("fixed", [False, True])
@pytest.mark.parametrize("n", [64, 128])
def test_block_egkb_matches_multikernel_path(n, fixed, monkeypatch):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    psf = _psf(900 + n)
    rank = 12 if fixed else 1e-3
    res = {}
    for name, env in (("block", None), ("multi", "0")):
        if env:
            monkeypatch.setenv("KPSB_EGKB_BLOCK", env)
        kp = K.kp_build(psf, n, 1, rank, K.EGKB, seed=4242)
        res[name] = (K.kp_info(kp), _vecs(K, kp))
        if env:
            monkeypatch.delenv("KPSB_EGKB_BLOCK")
    ib, (Ub, sb, Vb) = res["block"]
    im, (Um, sm, Vm) = res["multi"]
    assert ib["k"] == im["k"] and ib["kp"] == im["kp"]
    assert np.max(np.abs(sb - sm)) <= 2e-5 * sm[0]
    for i in range(min(4, ib["k"])):
        gap = min(abs(sm[i] - sm[i + 1]) if i + 1 < len(sm) else np.inf, abs(sm[i - 1] - sm[i]) if i else np.inf)
        if gap < 1e-2 * sm[0]:
            continue
        # a pair is unique up to a common sign; the sign convention picks it, except where the
        # largest entries of Ay_i tie in magnitude (symmetric PSFs), where rounding decides
        cu, cv = Ub[:, i] @ Um[:, i], Vb[:, i] @ Vm[:, i]
        assert abs(abs(cu) - 1) < 1e-3 and abs(abs(cv) - 1) < 1e-3 and cu * cv > 0


def test_block_egkb_batched_equals_alone():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    probs = []
    for i, n in enumerate([32, 64, 100, 128, 128, 72, 128, 96]):
        probs.append(dict(psf=_psf(50 + i, 31 if n >= 64 else 15), n=n, bc=i % 2,
                          rank_or_tol=1e-3 if i % 3 else 6, method=K.EGKB, seed=1000 + i,
                          one_sided=bool(i % 4 == 3)))
    batch = K.kp_build_batched(probs)
    for pr, kb in zip(probs, batch):
        ka = K.kp_build(pr["psf"], pr["n"], pr["bc"], pr["rank_or_tol"], K.EGKB, seed=pr["seed"],
                        one_sided=pr["one_sided"])
        Axa, Aya, sa = K.kp_get_factors(ka)
        Axb, Ayb, sb = K.kp_get_factors(kb)
        assert np.array_equal(sa, sb)
        assert np.array_equal(Axa, Axb) and np.array_equal(Aya, Ayb)


def test_block_egkb_breakdowns():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    n = 48
    # separable PSF: R(A) has rank 1, the recurrence breaks down after one step
    kp = K.kp_build(I.psf_separable(7, I.rng(2)), n, K.BC_REFLEXIVE, 3, K.EGKB, seed=3)
    assert K.kp_info(kp)["k"] == 1
    # rank(R(A)) <= s for a 5 x 5 PSF: k_p capped by the breakdown
    psf = I.psf_random(5, I.rng(5))
    kp = K.kp_build(psf, n, K.BC_ZERO, 4, K.EGKB, p=6, seed=7)
    inf = K.kp_info(kp)
    cf = O.r_sigma_closed_form(O.r_factors(psf, n, K.BC_ZERO))
    assert inf["k"] == 4 and inf["kp"] <= 5
    np.testing.assert_allclose(inf["sigma"], cf[:4], rtol=0, atol=1e-4 * cf[0])
    # a zero PSF: R(A) = 0, alpha_1 = 0, no accepted q: the build reports the breakdown
    with pytest.raises(Exception):
        K.kp_build(np.zeros((3, 3)), n, K.BC_ZERO, 2, K.EGKB, seed=1)
