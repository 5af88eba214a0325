"""R(A) index map, matrix-free R(A) apply, exact blur and the device Jacobi SVD vs the oracle."""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import dev_f32, dev_f64, host, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
@pytest.mark.parametrize("n,s0,s1", [(8, 5, 5), (16, 7, 4), (9, 3, 9), (20, 9, 7)])
def test_materialized_R_is_bit_exact(bc, n, s0, s1):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    # integer taps: every sum of taps is exact in FP32 and FP64, so the gather is bit-exact
    psf = np.arange(1, s0 * s1 + 1, dtype=np.float64).reshape(s0, s1)
    R = O.rearrange(O.blur_matrix(psf, n, bc), n, n, n, n)
    Rd = torch.zeros(n ** 4, dtype=torch.float32, device="cuda")
    K.kp_ra_materialize_dev(dev_f32(psf).data_ptr(), s0, s1, n, bc, Rd.data_ptr())
    got = host(Rd, (n * n, n * n))
    assert np.array_equal(got.astype(np.float64), R)


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
@pytest.mark.parametrize("n,s,nb", [(32, 9, 1), (100, 31, 3), (128, 31, 2), (70, 63, 1)])
@pytest.mark.parametrize("transpose", [0, 1])
def test_ra_apply_matches_oracle(bc, n, s, nb, transpose):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    g = I.rng(7 * n + s + bc + 100 * transpose)
    psf = I.psf_gaussian_mixture(s, g)
    psf[0, -1] += 0.02  # make P non-symmetric so R and R^T differ
    F = O.r_factors(psf, n, bc)
    V = g.standard_normal((n * n, nb)).astype(np.float32)
    ref = (O.r_apply_t if transpose else O.r_apply)(F, V.astype(np.float64))
    ld = n * n + 5  # padded leading dimension
    Vd = torch.zeros(ld * nb, dtype=torch.float32, device="cuda")
    for c in range(nb):
        Vd[c * ld:c * ld + n * n] = torch.from_numpy(V[:, c].copy()).cuda()
    Ud = torch.full((ld * nb,), 7.0, dtype=torch.float32, device="cuda")
    K.kp_ra_apply_dev(dev_f32(psf).data_ptr(), s, s, n, bc, Vd.data_ptr(), ld, nb, Ud.data_ptr(), ld,
                      transpose)
    torch.cuda.synchronize()
    U = Ud.cpu().numpy()
    for c in range(nb):
        got = U[c * ld:c * ld + n * n].astype(np.float64)
        err = np.linalg.norm(got - ref[:, c]) / np.linalg.norm(ref[:, c])
        assert err < 2e-6, err
        assert np.all(U[c * ld + n * n:(c + 1) * ld] == 7.0)  # padding untouched


@pytest.mark.parametrize("bc", [O.BC_ZERO, O.BC_REFLEXIVE])
@pytest.mark.parametrize("n,s", [(16, 5), (64, 15), (100, 9)])
@pytest.mark.parametrize("transpose", [0, 1])
def test_exact_blur_matches_oracle(bc, n, s, transpose):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    g = I.rng(3 * n + s + bc)
    psf = I.psf_random(s, g)
    X = g.uniform(size=(n, n))
    if transpose:
        if n > 20:
            pytest.skip("explicit transpose reference only at small n")
        ref = O.array(O.blur_matrix(psf, n, bc).T @ O.vec(X), n, n)
    else:
        ref = O.blur(psf, X, bc)
    Xd = dev_f64(X)
    Bd = torch.zeros_like(Xd)
    K.kp_blur_dev(dev_f64(psf).data_ptr(), s, s, n, bc, Xd.data_ptr(), Bd.data_ptr(), transpose)
    got = host(Bd, (n, n))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("m,nc,kind", [(11, 10, "bidiag"), (41, 40, "bidiag"), (64, 64, "dense"),
                                       (128, 64, "dense"), (30, 30, "psd"), (20, 12, "rankdef"),
                                       (1, 1, "dense"), (7, 3, "dense")])
def test_small_svd_matches_lapack(m, nc, kind):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    g = I.rng(m * 100 + nc)
    if kind == "bidiag":
        A = np.zeros((m, nc))
        for i in range(nc):
            A[i, i] = g.uniform(0.1, 2) * 0.7 ** i
            A[i + 1, i] = g.uniform(0.1, 2) * 0.7 ** i
    elif kind == "psd":
        Bm = g.standard_normal((nc, nc))
        A = Bm @ Bm.T
    elif kind == "rankdef":
        A = g.standard_normal((m, 5)) @ g.standard_normal((5, nc))
    else:
        A = g.standard_normal((m, nc))
    U, S, V, sweeps = K.kpsb_small_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(S, ref, rtol=0, atol=1e-13 * ref[0])
    assert np.all(np.diff(S) <= 0)
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, A, atol=1e-12 * ref[0])
    np.testing.assert_allclose(V.T @ V, np.eye(nc), atol=1e-12)
    r = int(np.sum(S > 1e-10 * S[0]))
    np.testing.assert_allclose(U[:, :r].T @ U[:, :r], np.eye(r), atol=1e-10)
    assert 1 <= sweeps <= 60
