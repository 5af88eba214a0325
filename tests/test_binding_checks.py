"""The Python binding checks every host array against the sizes the C ABI will read or write
before it calls the library, so a wrong shape raises ValueError instead of reading or
writing past a buffer (no GPU and no library call needed: the checks come first)."""
import numpy as np
import pytest

from paper_2410_00233_gb300 import kpsb as K


def _handle(n):
    return K.KP(0, n)  # a null handle that knows its image side; never reaches the library


@pytest.mark.parametrize("shape", [(4, 4), (8, 7), (64,), (8, 8, 1)])
def test_apply_and_solve_reject_wrong_image_shapes(shape):
    kp = _handle(8)
    with pytest.raises(ValueError):
        K.kp_apply(kp, np.zeros(shape))
    with pytest.raises(ValueError):
        K.sb_solve(kp, np.zeros(shape), 1.0, 0.1, K.ISO, 2)
    with pytest.raises(ValueError):
        K.sb_solve_batched([dict(kp=kp, b=np.zeros(shape), mu=1.0, lam=0.1, tv=K.ISO, iters=2)])


def test_factor_shapes_are_checked():
    k, n = 3, 8
    A = np.zeros((k, n, n), np.float32)
    with pytest.raises(ValueError):
        K.kp_from_factors(A, np.zeros((k, n, n - 1), np.float32), np.ones(k))
    with pytest.raises(ValueError):
        K.kp_from_factors(np.zeros((k, n, n + 1), np.float32), np.zeros((k, n, n + 1), np.float32), np.ones(k))
    with pytest.raises(ValueError):
        K.kp_from_factors(A, A, np.ones(k + 1))


def test_start_sizes_follow_the_method():
    n = 8
    psf = np.ones((3, 3)) / 9
    with pytest.raises(ValueError):  # EGKB: y has n^2 entries
        K.kp_build(psf, n, K.BC_ZERO, 4, K.EGKB, start=np.zeros(n * n - 1, np.float32))
    with pytest.raises(ValueError):  # RSVD: F is n^2 x (k + p)
        K.kp_build(psf, n, K.BC_ZERO, 4, K.RSVD, p=3, start=np.zeros((n * n, 6), np.float32))
    with pytest.raises(ValueError):  # RSVD with the default p = max(2, ceil(k/4)) = 2 for k = 5
        K.kp_build(psf, n, K.BC_ZERO, 5, K.RSVD, start=np.zeros((n * n, 8), np.float32))
    with pytest.raises(ValueError):
        K.kp_build_batched([dict(psf=psf, n=n, bc=K.BC_ZERO, rank_or_tol=4, start=np.zeros(3, np.float32))])


def test_start_size_rule_accepts_the_right_sizes():
    """The sizes the library reads pass the check (checked without calling the library)."""
    n = 8
    K._check_start(np.zeros(n * n), n, 4, K.EGKB, 0)
    K._check_start(np.zeros(n * n), n, 1e-3, K.EGKB, 4)  # automatic rank: y is still n^2
    K._check_start(np.zeros((n * n, 7)), n, 4, K.RSVD, 3)
    K._check_start(np.zeros((n * n, 7)), n, 5, K.RSVD, 0)  # 5 + max(2, 2)
    K._check_start(np.zeros((n * n, 20)), n, 16, K.RSVD, 0)  # 16 + max(2, 4)


def test_psf_must_be_two_dimensional():
    with pytest.raises(ValueError):
        K.kp_build(np.ones(9), 8, K.BC_ZERO, 2, K.EGKB)
    with pytest.raises(ValueError):
        K.kp_dense_blur(np.ones((0, 3)), 8, K.BC_ZERO)


def test_batched_build_frees_the_built_handles_when_one_problem_fails(monkeypatch):
    """kp_build_batched returns the first error but still builds the other problems; the
    binding frees those handles before it raises (a fake library stands in for the C ABI)."""
    freed = []

    class FakeLib:
        def kp_build_batched(self, count, arr, outs):
            outs[0], outs[1], outs[2] = 0x1000, None, 0x2000  # problem 1 failed
            return -1

        def kp_free(self, ptr):
            freed.append(ptr.value)

        def kpsb_last_error(self):
            return b"problem 1: rank 0 outside [1, 64]"

    monkeypatch.setattr(K, "lib", lambda: FakeLib())
    psf = np.ones((3, 3)) / 9
    probs = [dict(psf=psf, n=8, bc=K.BC_ZERO, rank_or_tol=4) for _ in range(3)]
    with pytest.raises(K.KpsbError) as e:
        K.kp_build_batched(probs)
    assert e.value.code == -1 and "problem 1" in str(e.value)
    assert sorted(freed) == [0x1000, 0x2000]
