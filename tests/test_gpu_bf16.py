"""BF16 split-precision KP GEMMs (tcgen05 kind::f16, FP32 accumulation) and the tensor-core
path at image sides that are not a multiple of the 128-row tile, against the oracle.

BF16X2 uses the factors rounded once to BF16 (sigma folded in FP32 first): against the
oracle applied with those same rounded factors only the split of the image (two BF16 parts,
2^-18 relative), the split intermediate and the FP32 accumulation remain: bound 1e-4
relative.  BF16X3 splits both operands in two BF16 parts and drops the lo*lo product
(2^-18 relative per product): against the FP32 factors the bound is 1e-4.  The TF32 modes
keep their own bounds (1e-4 TF32X3; 1e-4 TF32X2 against its rounded factors) at the
masked sizes.
"""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round to BF16 (8 significant bits), to nearest with ties to even (finite values)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def _tf32(a):
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


def _rand_factors(n, k, seed):
    g = I.rng(seed)
    Ax = g.standard_normal((k, n, n)).astype(np.float32)
    Ay = g.standard_normal((k, n, n)).astype(np.float32)
    for i in range(k):
        Ax[i] /= np.linalg.norm(Ax[i])
        Ay[i] /= np.linalg.norm(Ay[i])
    sig = np.sort(g.uniform(0.1, 3.0, size=k))[::-1].copy()
    return Ax, Ay, sig


def _op(Ax, Ay, sig, rnd=None):
    k = Ax.shape[0]
    sx = np.stack([np.float32(sig[i]) * Ax[i] for i in range(k)])
    if rnd is not None:
        sx, Ay = rnd(sx), rnd(Ay)
    return O.KPSum(Ax=sx.astype(np.float64), Ay=np.asarray(Ay).astype(np.float64), sigma=np.ones(k))


@pytest.mark.parametrize("n,k", [(64, 5), (100, 3), (128, 12), (200, 7), (256, 1), (384, 4), (512, 3), (640, 2)])
@pytest.mark.parametrize("transpose", [0, 1])
def test_kp_apply_bf16_modes(n, k, transpose):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    Ax, Ay, sig = _rand_factors(n, k, 13 * n + k)
    kp = K.kp_from_factors(Ax, Ay, sig)
    X = I.rng(9 + k).standard_normal((n, n))
    ap = O.kp_apply_t if transpose else O.kp_apply
    ref32 = ap(_op(Ax, Ay, sig), X)
    ref_b = ap(_op(Ax, Ay, sig, _bf16), X)
    y3 = K.kp_apply(kp, X, transpose, K.P_BF16X3)
    y2 = K.kp_apply(kp, X, transpose, K.P_BF16X2)
    e3 = np.linalg.norm(y3 - ref32) / np.linalg.norm(ref32)
    e2 = np.linalg.norm(y2 - ref_b) / np.linalg.norm(ref_b)
    assert e3 < 1e-4, e3
    assert e2 < 1e-4, e2
    # element-wise: no tile garbage in the masked rows and columns
    assert np.abs(y3 - ref32).max() <= 1e-3 * np.abs(ref32).max()
    assert np.abs(y2 - ref_b).max() <= 1e-3 * np.abs(ref_b).max()
    # BF16X2's rounded factors move the operator by ~2^-9 relative
    assert np.linalg.norm(y2 - ref32) / np.linalg.norm(ref32) < 1e-2


@pytest.mark.parametrize("n,k", [(64, 5), (100, 3), (200, 7), (520, 2), (1024, 2)])
@pytest.mark.parametrize("transpose", [0, 1])
def test_kp_apply_tf32_modes_at_masked_sizes(n, k, transpose):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    Ax, Ay, sig = _rand_factors(n, k, 17 * n + k)
    kp = K.kp_from_factors(Ax, Ay, sig)
    X = I.rng(3 + k).standard_normal((n, n))
    ap = O.kp_apply_t if transpose else O.kp_apply
    ref32 = ap(_op(Ax, Ay, sig), X)
    ref_t = ap(_op(Ax, Ay, sig, _tf32), X)
    y3 = K.kp_apply(kp, X, transpose, K.P_TF32X3)
    y2 = K.kp_apply(kp, X, transpose, K.P_TF32X2)
    assert np.linalg.norm(y3 - ref32) / np.linalg.norm(ref32) < 1e-4
    assert np.linalg.norm(y2 - ref_t) / np.linalg.norm(ref_t) < 1e-4
    assert np.abs(y3 - ref32).max() <= 5e-4 * np.abs(ref32).max()


def test_bf16_and_masked_apply_count_their_work():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    for n, k, prec in ((100, 3, K.P_BF16X3), (64, 4, K.P_TF32X2), (256, 2, K.P_BF16X2)):
        Ax, Ay, sig = _rand_factors(n, k, n + 5 * k)
        kp = K.kp_from_factors(Ax, Ay, sig)
        X = I.rng(1).standard_normal((n, n))
        K.kpsb_gemm_timing(True)
        try:
            K.kp_apply(kp, X, 0, prec)
            assert K.kpsb_apply_counts() == (1, k * n ** 3)
        finally:
            K.kpsb_gemm_timing(False)


@pytest.mark.parametrize("prec_name,sizes", [("P_BF16X3", (512, 512, 640)), ("P_BF16X3", (256, 384)),
                                             ("P_TF32X2", (1024, 520))])
def test_split_stage2_batched_equals_alone(prec_name, sizes):
    """The two-stage apply's stage 2 splits K into ranges fixed by n where it is the only
    variant (BF16 modes; TF32 at n > 384 or n not a multiple of 128) and the tile's last CTA
    adds the partial tiles in range order: problems with different k in one batched solve give
    the bits of their solves alone, and the apply stays within the oracle bounds above."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    prec = getattr(K, prec_name)
    jobs, alone = [], []
    for i, n in enumerate(sizes):
        k = 2 + 2 * i
        Ax, Ay, sig = _rand_factors(n, k, 7700 + 10 * n + i)
        kp = K.kp_from_factors(Ax, Ay, sig)
        X = I.rng(31 + i).standard_normal((n, n))
        rnd = _tf32 if prec_name == "P_TF32X2" else None
        ref = O.kp_apply(_op(Ax, Ay, sig, rnd), X)
        y = K.kp_apply(kp, X, 0, prec)
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-4, (n, k)
        b = I.rng(77 + i).uniform(0.0, 1.0, (n, n))
        x, st = K.sb_solve(kp, b, 1.0, 0.1, K.ISO, 2, i_max=3, fixed_inner=True, prec=prec)
        alone.append(x)
        jobs.append(dict(kp=kp, b=b, mu=1.0, lam=0.1, tv=K.ISO, iters=2))
    outs, _ = K.sb_solve_batched(jobs, prec=prec, i_max=3, fixed_inner=True)
    for x, xb in zip(alone, outs):
        assert np.array_equal(x, xb)
