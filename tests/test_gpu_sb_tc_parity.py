"""Element-wise parity of the tensor-core split Bregman path with the oracle (Alg. 3-5).

The mixed path (KPSB_P_TF32X2 / KPSB_P_TF32X3) applies the KP sum on the tensor cores and
keeps every CGLS vector, update and ||f||^2 in FP64; the sums of squares of FP32 values are
taken in FP32 per thread: ||z||^2 = mu ||z1||^2 + (lambda/2)^2 ||D w_f||^2 of the vector the
apply saw (w_f = fl32(w), z1 its FP32 product), and ||w_f||^2, ||fl32(x)||^2 of RC_CGLS.
The TV rows r2, r3 of the residual are carried as q = Dx^T r2 + Dy^T r3 (the only way they
enter step 7), updated by the image of step 6 on the FP32 direction w_f, as the data row is
(z1 = A w_f): the same iteration in exact arithmetic, ~1e-7 |w| per step besides.
Against the oracle run on the SAME rounded operator, what is left is per-apply rounding:
the iterate rounded to FP32 and split in two TF32 parts (2^-22 relative), the split
intermediate (2^-22), the tensor-core FP32 accumulation (about sqrt(K) 2^-24, K <= 1536
here) and the FP32 output (2^-24): a per-apply relative error e_a of a few 1e-6 for these
smooth, positive operators.  Split Bregman with a fixed inner count turns a per-apply
relative perturbation e_a into at most ~5 e_a of max|x| element-wise over 3 outer x 10 inner
steps (measured on the CPU by perturbing the oracle's own applies at n = 128 and 256), i.e.
~1e-5; the bounds keep a factor 10: 1e-4 of max|x| element-wise and 5e-5 relative in the
Frobenius norm.  The BF16 modes split in two BF16 parts (2^-18 relative for the image and the
intermediate, and BF16X3 drops the lo*lo product, 2^-18): e_a ~6e-6, bounds 3e-4 and 1e-4.
n = 200 runs the masked two-stage kernel.  (Measured on GB300: at most 3.3e-6 element-wise
for the TF32 modes and 7.9e-6 for the BF16 modes.)

The rounded operators:
  TF32X2: Ax_i' = tf32(fl32(sigma_i) * Ax_i), Ay_i' = tf32(Ay_i), sigma' = 1 (the tables the
          kernels read; tf32 = round to nearest, ties away, 10 explicit mantissa bits);
  BF16X2: the same with bf16 (round to nearest even, 8 significant bits);
  TF32X3, BF16X3: Ax_i' = fl32(fl32(sigma_i) * Ax_i), Ay_i' = Ay_i (FP32-class products).
The factors come from the oracle's own TSVD (Alg. 1) of a synthetic PSF, rounded to FP32.
The FP64 path is held to 1e-10 at the headline size n = 128 (8 reduction chunks).
"""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

MU, LAM = 1.0, 0.1
BETA = LAM * LAM / 2.0


def _tf32(a):
    """Round to TF32 (10 explicit mantissa bits), to nearest with ties away from zero."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


_CACHE = {}


def _problem(n, seed):
    """Blurred data and FP32 KP factors of the oracle's EGKB (k = 6, p = 3) for a 31 x 31
    two-Gaussian mixture PSF with reflexive boundary, 1 % noise."""
    key = (n, seed)
    if key not in _CACHE:
        g = I.rng(seed)
        psf = I.psf_gaussian_mixture(31, g)
        x_true = I.image_piecewise_constant(n, g)
        bt = O.blur(psf, x_true, 1)
        b = bt + I.noise_vector(bt, 0.01, I.gaussian((n, n), g))
        F = O.r_factors(psf, n, 1)
        ts = O.egkb(lambda v: O.r_apply(F, v), lambda u: O.r_apply_t(F, u), I.gaussian(n * n, g), 6, 3)
        Kop = O.kp_terms(ts, n)
        _CACHE[key] = (x_true, b, Kop.Ax.astype(np.float32), Kop.Ay.astype(np.float32), Kop.sigma)
    return _CACHE[key]


def _bf16(a):
    """Round to BF16 (8 significant bits), to nearest with ties to even (finite values)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def _rounded_operator(Ax, Ay, sig, prec_name):
    k = Ax.shape[0]
    sx = [np.float32(sig[i]) * Ax[i] for i in range(k)]  # sigma folded in FP32, as the tables do
    rnd = {"P_TF32X2": _tf32, "P_BF16X2": _bf16}.get(prec_name)
    if rnd is not None:
        Axr = np.stack([rnd(a) for a in sx]).astype(np.float64)
        Ayr = rnd(Ay).astype(np.float64)
    else:
        Axr = np.stack(sx).astype(np.float64)
        Ayr = Ay.astype(np.float64)
    return O.KPSum(Ax=Axr, Ay=Ayr, sigma=np.ones(k))


_BOUNDS = {"P_TF32X2": (1e-4, 5e-5), "P_TF32X3": (1e-4, 5e-5), "P_BF16X3": (3e-4, 1e-4),
           "P_BF16X2": (3e-4, 1e-4)}


@pytest.mark.parametrize("prec_name", ["P_TF32X2", "P_TF32X3", "P_BF16X3", "P_BF16X2"])
@pytest.mark.parametrize("iso", [False, True])
@pytest.mark.parametrize("n", [128, 256, 200])
def test_tensor_core_sb_matches_oracle_elementwise(n, iso, prec_name):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    x_true, b, Ax, Ay, sig = _problem(n, 900 + n)
    kp = K.kp_from_factors(Ax, Ay, sig)
    op = _rounded_operator(Ax, Ay, sig, prec_name)
    iters, i_max = 3, 10
    x, st = K.sb_solve(kp, b, MU, LAM, K.ISO if iso else K.ANISO, iters, i_max=i_max, fixed_inner=True,
                       prec=getattr(K, prec_name))
    ref = O.split_bregman(lambda X: O.kp_apply(op, X), lambda Y: O.kp_apply_t(op, Y), b, MU, LAM, BETA, iso,
                          iters, i_max=i_max, fixed_inner=True)
    assert st.l_end == iters and st.iota_total == iters * i_max
    scale = np.abs(ref.x).max()
    err_max = np.abs(x - ref.x).max() / scale
    err_fro = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    b_max, b_fro = _BOUNDS[prec_name]
    assert err_max < b_max, (err_max, err_fro)
    assert err_fro < b_fro, (err_max, err_fro)
    # the outer stopping quantity follows the same iterates
    assert abs(st.rc_sb - ref.rc_sb) <= 1e-3 * ref.rc_sb


@pytest.mark.parametrize("iso", [False, True])
def test_fp64_sb_matches_oracle_at_n128(iso):
    """The FP64 path at the headline size (16384 pixels: 8 fixed 2048-element reduction
    chunks per vector) within 1e-10 of the oracle on identical factors."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    x_true, b, Ax, Ay, sig = _problem(128, 1028)
    kp = K.kp_from_factors(Ax, Ay, sig)
    op = O.KPSum(Ax=Ax.astype(np.float64), Ay=Ay.astype(np.float64), sigma=np.asarray(sig, dtype=np.float64))
    for iters, i_max in ((1, 1), (4, 12)):
        x, st = K.sb_solve(kp, b, MU, LAM, K.ISO if iso else K.ANISO, iters, i_max=i_max, fixed_inner=True,
                           prec=K.P_FP64)
        ref = O.split_bregman(lambda X: O.kp_apply(op, X), lambda Y: O.kp_apply_t(op, Y), b, MU, LAM, BETA,
                              iso, iters, i_max=i_max, fixed_inner=True)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-10
        assert np.abs(x - ref.x).max() <= 1e-10 * np.abs(ref.x).max()
        assert st.iota_total == iters * i_max
        assert abs(st.rc_sb - ref.rc_sb) <= 1e-8 * ref.rc_sb


@pytest.mark.parametrize("prec_name", ["P_TF32X2", "P_BF16X3"])
def test_tensor_core_sb_matches_oracle_elementwise_n1024(prec_name):
    """The largest serving size: 256-column stage-1 tiles, split planes written by the vector
    kernels, FP32 apply results; same bounds as above."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    n = 1024
    x_true, b, Ax, Ay, sig = _problem(n, 1900)
    kp = K.kp_from_factors(Ax, Ay, sig)
    op = _rounded_operator(Ax, Ay, sig, prec_name)
    x, st = K.sb_solve(kp, b, MU, LAM, K.ISO, 2, i_max=6, fixed_inner=True, prec=getattr(K, prec_name))
    ref = O.split_bregman(lambda X: O.kp_apply(op, X), lambda Y: O.kp_apply_t(op, Y), b, MU, LAM, BETA, True,
                          2, i_max=6, fixed_inner=True)
    b_max, b_fro = _BOUNDS[prec_name]
    err_max = np.abs(x - ref.x).max() / np.abs(ref.x).max()
    err_fro = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    assert err_max < b_max and err_fro < b_fro, (err_max, err_fro)
