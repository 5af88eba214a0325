"""The integer binary32 <-> binary64 conversions of the split Bregman vector kernels give the
bits of the hardware conversions: every binary32 value widened, and random binary64 values
(binary32 subnormal / normal / overflow range, round-to-nearest-even ties, zeros,
infinities, NaNs) rounded."""
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2])
def test_integer_conversions_match_hardware(seed):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    assert K.kpsb_conversion_check(1 << 27, seed) == 0
