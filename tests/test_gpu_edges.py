"""Edge and degenerate cases of the GPU path against what the mathematics fixes: empty
batches, the identity blur (1 x 1 PSF), a PSF larger than the image, a non-square PSF, zero
data, and the largest image side the workloads use (n = 1024)."""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_empty_batches_return_empty():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    assert K.kp_build_batched([]) == []
    outs, stats = K.sb_solve_batched([])
    assert outs == [] and stats == []


@pytest.mark.parametrize("n", [2, 8])
def test_identity_psf_gives_one_term_with_sigma_n(n):
    """A 1 x 1 PSF is the identity: A = I (x) I, so R(A) = vec(I) vec(I)^T has exactly one
    singular value, ||vec(I)||^2 = n; the build stops at k = 1 (breakdown) with that value."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    for bc in (K.BC_ZERO, K.BC_REFLEXIVE):
        kp = K.kp_build(np.ones((1, 1)), n, bc, 3, K.EGKB, seed=1)
        inf = K.kp_info(kp)
        assert inf["k"] == 1 and abs(inf["sigma"][0] - n) <= 1e-5 * n
        X = I.rng(n).standard_normal((n, n))
        assert np.allclose(K.kp_apply(kp, X, 0, K.P_FP64), X, rtol=0, atol=1e-6 * np.abs(X).max())


def test_identity_blur_split_bregman_is_tv_denoising():
    """With A = I split Bregman is TV denoising: the FP64 path equals the oracle run on the
    identity operator to 1e-10 (fixed inner counts)."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    n = 16
    g = I.rng(12)
    x_true = I.image_piecewise_constant(n, g)
    b = x_true + I.noise_vector(x_true, 0.05, I.gaussian((n, n), g))
    kp = K.kp_build(np.ones((1, 1)), n, K.BC_ZERO, 1, K.EGKB, seed=1)
    Ax, Ay, sig = K.kp_get_factors(kp)
    Kop = O.KPSum(Ax=Ax.astype(np.float64), Ay=Ay.astype(np.float64), sigma=sig)
    x, st = K.sb_solve(kp, b, 1.0, 0.3, K.ISO, 3, i_max=10, fixed_inner=True)
    ref = O.split_bregman(lambda X: O.kp_apply(Kop, X), lambda Y: O.kp_apply_t(Kop, Y), b, 1.0, 0.3,
                          0.045, True, 3, i_max=10, fixed_inner=True)
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("n,s0,s1", [(5, 9, 9), (12, 7, 4), (10, 3, 11)])
def test_psf_larger_than_image_or_non_square(n, s0, s1):
    """Zero boundary with a PSF wider than the image, and non-square PSFs: the leading
    singular values of the build equal the closed form sigma(Gx^1/2 P^T Gy^1/2)."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    psf = I.rng(s0 * 31 + s1).random((s0, s1))
    psf /= psf.sum()
    ref = O.r_sigma_closed_form(O.r_factors(psf, n, O.BC_ZERO))
    k = min(3, int(np.sum(ref > 1e-6 * ref[0])))
    kp = K.kp_build(psf, n, K.BC_ZERO, k, K.EGKB, p=3, seed=4)
    sig = K.kp_info(kp)["sigma"]
    kk = min(len(sig), k)
    assert np.max(np.abs(sig[:kk] - ref[:kk])) <= 1e-4 * ref[0]


def test_zero_data_gives_zero_image():
    """b = 0: Ahat^T bhat = 0 at every outer step, so CGLS stops at once and x = 0 exactly,
    with no division by zero (RC_CGLS uses the updated iterate)."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    pr = I.problem_small(2)
    kp = K.kp_build(pr.psf, pr.n, pr.bc, 5, K.EGKB, p=4, seed=2)
    for prec in (K.P_FP64, K.P_FP32):
        x, st = K.sb_solve(kp, np.zeros((pr.n, pr.n)), 1.0, 0.1, K.ANISO, 3, prec=prec)
        assert np.all(x == 0.0) and st.iota_total == 0 and st.l_end == 3
    assert np.all(K.kp_apply(kp, np.zeros((pr.n, pr.n)), 0, K.P_FP64) == 0.0)


def test_largest_size_build_and_tensor_core_apply():
    """n = 1024 (the serving configuration's largest side): the build's leading sigma_k
    against the closed form, and one TF32x3 apply of random factors against the oracle."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    n = 1024
    psf = I.psf_gaussian(15, 2.0, 3.5, 20.0)
    ref = O.r_sigma_closed_form(O.r_factors(psf, n, O.BC_REFLEXIVE))
    kp = K.kp_build(psf, n, K.BC_REFLEXIVE, 4, K.EGKB, p=4, seed=6)
    sig = K.kp_info(kp)["sigma"]
    assert np.max(np.abs(sig - ref[:4])) <= 1e-4 * ref[0]
    g = I.rng(99)
    k = 2
    Ax = (g.standard_normal((k, n, n)) / n).astype(np.float32)
    Ay = (g.standard_normal((k, n, n)) / n).astype(np.float32)
    s = np.array([1.0, 0.5])
    op = O.KPSum(Ax=Ax.astype(np.float64), Ay=Ay.astype(np.float64), sigma=s)
    X = g.standard_normal((n, n))
    kp2 = K.kp_from_factors(Ax, Ay, s)
    for t in (0, 1):
        ref_y = O.kp_apply_t(op, X) if t else O.kp_apply(op, X)
        y = K.kp_apply(kp2, X, t, K.P_TF32X3)
        assert np.linalg.norm(y - ref_y) <= 1e-4 * np.linalg.norm(ref_y), t


def test_bounded_wait_times_out_and_the_device_stays_usable():
    """The tensor-core pipelines bound every mbarrier wait; a wait that runs out records an
    error flag that the host maps to KPSB_ETIMEOUT.  The self-test drives that branch with a
    wait on an mbarrier nothing arrives at (a limit of microseconds, not the pipelines' one
    second); afterwards the flag is clear and an apply on the same device is still exact."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    for limit_us in (20, 200):
        with pytest.raises(K.KpsbError) as e:
            K.kpsb_wait_selftest(limit_us)
        assert e.value.code == -4 and "timed out" in str(e.value)
    with pytest.raises(K.KpsbError) as e:
        K.kpsb_wait_selftest(0)
    assert e.value.code == -1
    n, k = 128, 3
    g = I.rng(17)
    Ax = g.standard_normal((k, n, n)).astype(np.float32)
    Ay = g.standard_normal((k, n, n)).astype(np.float32)
    sig = np.array([2.0, 1.0, 0.5])
    kp = K.kp_from_factors(Ax, Ay, sig)
    X = g.standard_normal((n, n))
    ref = O.kp_apply(O.KPSum(Ax=Ax.astype(np.float64), Ay=Ay.astype(np.float64), sigma=sig), X)
    y = K.kp_apply(kp, X, 0, K.P_TF32X3)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-4
