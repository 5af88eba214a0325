"""Direct split Bregman with the explicit blurring operator A (the paper's comparison path,
Sec. 4.3 case (i)): the dense operator against the oracle's explicit A, and split Bregman with
it against the oracle's split Bregman run on the same A."""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n,s", [(16, 5), (20, 7), (33, 9)])
def test_explicit_operator_matches_oracle_matrix(n, s, bc):
    """A x and A^T x through the explicit-operator handle equal the oracle's explicit A
    (eq. (1.1)) applied to the same x (FP64; ragged n, both boundary conditions)."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    g = I.rng(3 * n + s + bc)
    psf = I.psf_gaussian(s, 1.2, 2.1, 0.4) if s > 5 else g.random((s, s))
    psf = psf / psf.sum()
    A = O.blur_matrix(psf, n, bc)
    kp = K.kp_dense_blur(psf, n, bc)
    X = g.standard_normal((n, n))
    for t in (0, 1):
        ref = ((A.T if t else A) @ X.reshape(-1, order="F")).reshape(n, n, order="F")
        y = K.kp_apply(kp, X, t, K.P_FP64)
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref), t
    assert K.kp_info(kp)["k"] == 0
    with pytest.raises(K.KpsbError):
        K.kp_get_factors(kp)
    with pytest.raises(K.KpsbError):
        K.kp_apply(kp, X, 0, K.P_TF32X2)


@pytest.mark.parametrize("iso", [False, True])
def test_direct_split_bregman_matches_oracle(iso):
    """Split Bregman with the explicit A (FP64) equals the oracle's split Bregman with the
    same A to 1e-10 with fixed inner counts."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    pr = I.problem_small(4)
    n = pr.n
    bt = O.blur(pr.psf, pr.x_true, pr.bc)
    b = bt + I.noise_vector(bt, pr.eta, pr.zeta)
    A = O.blur_matrix(pr.psf, n, pr.bc)
    kp = K.kp_dense_blur(pr.psf, n, pr.bc)
    mu, lam = 1.0, 0.1
    x, st = K.sb_solve(kp, b, mu, lam, K.ISO if iso else K.ANISO, 3, i_max=12, fixed_inner=True)
    fwd = lambda X: (A @ X.reshape(-1, order="F")).reshape(n, n, order="F")  # noqa: E731
    adj = lambda Y: (A.T @ Y.reshape(-1, order="F")).reshape(n, n, order="F")  # noqa: E731
    ref = O.split_bregman(fwd, adj, b, mu, lam, lam * lam / 2.0, iso, 3, i_max=12, fixed_inner=True)
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    assert st.iota_total == 36


def test_explicit_and_kp_jobs_in_one_batch_equal_alone():
    """A batch mixing explicit-operator and Kronecker-sum handles (same and different n)
    groups them by operator kind; every job equals its solve alone, bit for bit."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    jobs, alone = [], []
    for i, n in enumerate((32, 32, 48)):
        pr = I.problem_small(10 + i)
        psf = pr.psf
        x_true = pr.x_true if n == pr.n else I.image_piecewise_constant(n, I.rng(60 + i))
        bt = O.blur(psf, x_true, pr.bc)
        b = bt + I.noise_vector(bt, 0.01, I.gaussian((n, n), I.rng(70 + i)))
        dense = K.kp_dense_blur(psf, n, pr.bc)
        kp = K.kp_build(psf, n, pr.bc, 5, K.EGKB, p=4, seed=9 + i)
        for h in (dense, kp):
            jobs.append(dict(kp=h, b=b, mu=1.0, lam=0.1, tv=K.ANISO, iters=2))
            alone.append(K.sb_solve(h, b, 1.0, 0.1, K.ANISO, 2))
    outs, stats = K.sb_solve_batched(jobs)
    for (x, st), xb, sb in zip(alone, outs, stats):
        assert np.array_equal(x, xb) and st.iota_total == sb.iota_total


def _kron_operator(n, g, c=(5.0, 2.0, 1.0, 0.5), noise=1e-3):
    """A general (non-PSF) operator: a short sum of Kronecker products plus a dense
    perturbation, so R(A) has a clear leading rank-4 part and a noise floor."""
    A = sum(ci * np.kron(g.standard_normal((n, n)), g.standard_normal((n, n))) for ci in c)
    return A + noise * g.standard_normal(A.shape)


@pytest.mark.parametrize("method", ["EGKB", "RSVD"])
def test_general_operator_kp_build_matches_svd_of_rearrangement(method):
    """kp_build_dense on an explicit operator without PSF structure: the leading singular
    values equal those of the oracle's rearrangement R(A) (eq. (2.2)) from LAPACK, and the
    rank-4 KP sum equals the best rank-4 approximation built from that SVD (Thm 2.1), within
    single-precision tolerance."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    n, k = 16, 4
    A = _kron_operator(n, I.rng(41))
    R = O.rearrange(A, n, n, n, n)
    U, S, Vt = np.linalg.svd(R)
    kp = K.kp_build_dense(A, n, k, getattr(K, method), p=6, seed=5)
    Ax, Ay, sig = K.kp_get_factors(kp)
    assert np.max(np.abs(sig - S[:k])) <= 1e-4 * S[0]
    best = sum(S[i] * np.kron(U[:, i].reshape(n, n, order="F"), Vt[i].reshape(n, n, order="F"))
               for i in range(k))
    got = sum(sig[i] * np.kron(Ax[i].astype(np.float64), Ay[i].astype(np.float64)) for i in range(k))
    assert np.linalg.norm(got - best) <= 1e-4 * np.linalg.norm(A)


@pytest.mark.parametrize("bc", [0, 1])
def test_explicit_blur_kp_build_matches_closed_form(bc):
    """The explicit blur matrix through kp_build_dense has the singular values of the PSF's
    closed form sigma(Gx^1/2 P^T Gy^1/2), the same as the index-map path."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    pr = I.problem_small(7)
    n = pr.n
    A = O.blur_matrix(pr.psf, n, bc)
    ref = O.r_sigma_closed_form(O.r_factors(pr.psf, n, bc))
    kp = K.kp_build_dense(A, n, 5, K.EGKB, p=4, seed=2)
    sig = K.kp_info(kp)["sigma"]
    assert np.max(np.abs(sig - ref[:5])) <= 1e-4 * ref[0]
    kp2 = K.kp_build(pr.psf, n, bc, 5, K.EGKB, p=4, seed=2)
    assert np.max(np.abs(K.kp_info(kp2)["sigma"] - sig)) <= 1e-4 * ref[0]
