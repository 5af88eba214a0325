"""Helpers of the GPU tests: device buffers (torch) and column-major conversions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00233_gb300 import kpsb as K

    K.lib()  # loud failure if the library is missing


def dev_f64(a):
    """Device FP64 copy of a (column-major flattening)."""
    return torch.from_numpy(np.asarray(a, dtype=np.float64).reshape(-1, order="F").copy()).cuda()


def dev_f32(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32).reshape(-1, order="F").copy()).cuda()


def host(t, shape):
    torch.cuda.synchronize()
    return t.cpu().numpy().reshape(shape, order="F")
