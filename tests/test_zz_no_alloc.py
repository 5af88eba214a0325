"""The allocation-free R(A) block apply (kp_ra_apply_noalloc_dev) against kp_ra_apply_dev.

kp_ra_apply_noalloc_dev serves callers that cannot allocate device memory inside a call
(real-time loops that must not be stalled by cudaMalloc/cudaFree, or programs whose device
memory all belongs to their own pool).  Its scratch is a fixed array shared by every call,
so this test makes two different calls in a row and checks each against the allocating
entry point, then checks that an oversized request is refused.  This file is collected
last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import dev_f32, need_gpu, torch

pytestmark = pytest.mark.gpu


def _apply(K, fn, psf_d, s, n, bc, V, transpose):
    nb = V.shape[1]
    Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda().reshape(-1)
    Ud = torch.full((n * n * nb,), float("nan"), dtype=torch.float32, device="cuda")
    fn(psf_d.data_ptr(), s, s, n, bc, Vd.data_ptr(), n * n, nb, Ud.data_ptr(), n * n, transpose)
    torch.cuda.synchronize()
    return Ud.cpu().numpy().reshape(nb, n * n).T.astype(np.float64)


def test_noalloc_matches_allocating_apply_on_two_calls_in_a_row():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    cases = [(128, 31, K.BC_REFLEXIVE, 3, 0), (64, 15, K.BC_ZERO, 5, 1)]
    for call, (n, s, bc, nb, transpose) in enumerate(cases):
        g = I.rng(500 + call)
        psf = I.psf_gaussian_mixture(s, g)
        psf[0, -1] += 0.01
        psf_d = dev_f32(psf)
        V = g.standard_normal((n * n, nb)).astype(np.float32)
        ref = _apply(K, K.kp_ra_apply_dev, psf_d, s, n, bc, V, transpose)
        got = _apply(K, K.kp_ra_apply_noalloc_dev, psf_d, s, n, bc, V, transpose)
        assert np.all(np.isfinite(got))
        # same tolerance as the R(A) parity tests (FP32 apply), on top of identical kernels
        for c in range(nb):
            assert np.linalg.norm(got[:, c] - ref[:, c]) <= 2e-6 * np.linalg.norm(ref[:, c])
        F = O.r_factors(psf.astype(np.float32).astype(np.float64), n, bc)
        exact = (O.r_apply_t if transpose else O.r_apply)(F, V.astype(np.float64))
        for c in range(nb):
            assert np.linalg.norm(got[:, c] - exact[:, c]) <= 2e-6 * np.linalg.norm(exact[:, c])


def test_noalloc_refuses_requests_beyond_its_scratch():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    n, s, nb = 1024, 9, 16  # needs more than the fixed 4 MiB
    psf_d = dev_f32(np.ones((s, s), dtype=np.float32) / (s * s))
    V = torch.zeros(n * n * nb, dtype=torch.float32, device="cuda")
    U = torch.zeros_like(V)
    with pytest.raises(K.KpsbError) as e:
        K.kp_ra_apply_noalloc_dev(psf_d.data_ptr(), s, s, n, K.BC_ZERO, V.data_ptr(), n * n, nb,
                                  U.data_ptr(), n * n, 0)
    assert e.value.code == -1 and "scratch" in str(e.value)
