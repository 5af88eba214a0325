"""The KP apply's roofline classification in bench.py (host arithmetic, no GPU).

Per problem and apply the kernel reads two n x n factor tables per term (one plane for the
x2 modes, two for the x3 modes; 4 bytes per element in TF32, 2 in BF16), the two planes of the
split iterate and writes the FP32 result; the useful work is 4 k n^3 flops (Sec. 4.2).  Worked
by hand: TF32x2 at n = 128 with k = 6.35 moves 8 k n^2 + 12 n^2 bytes for 4 k n^3 flops,
51.8 flop/byte, below its ridge (833.26/2 TFLOP/s over 6784.5 GB/s = 61.4): HBM-bound.  BF16X3
at n = 1024, k = 20: 8 k n^2 + 8 n^2 bytes, 487.6 flop/byte, far above 1741/3 over 6784.5
(85.5): tensor-bound.
"""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _case(mode, n, k, problems, secs, peak, hbm):
    kn3 = problems * k * float(n) ** 3
    flops = 4.0 * kn3
    return bench.apply_roofline(mode, n, problems, kn3, flops, secs, peak, hbm)


def test_tf32x2_headline_is_hbm_bound():
    r = _case("tf32x2", 128, 6.35, 194, 66e-6, 833.26, 6784.5)
    nn = 128.0 * 128
    assert math.isclose(r["bytes"], 194 * (6.35 * 8 * nn + 12 * nn), rel_tol=1e-12)
    assert math.isclose(r["intensity"], 4 * 6.35 * 128 / (8 * 6.35 + 12), rel_tol=1e-12)
    assert math.isclose(r["ridge"], 833.26 / 2 * 1e3 / 6784.5, rel_tol=1e-12)
    assert r["bound"] == "hbm" and 51.7 < r["intensity"] < 51.9
    assert math.isclose(r["achieved_gbs"], r["bytes"] / 66e-6 / 1e9, rel_tol=1e-12)


def test_bf16x3_large_is_tensor_bound():
    r = _case("bf16x3", 1024, 20, 1, 150e-6, 1741.0, 6784.5)
    nn = 1024.0 * 1024
    assert math.isclose(r["bytes"], 20 * 2 * nn * 2 * 2 + (2 * nn * 2 + 4 * nn), rel_tol=1e-12)
    assert r["bound"] == "tensor" and r["intensity"] > 400 > r["ridge"] > 80


@pytest.mark.parametrize("mode,planes,es", [("tf32x2", 1, 4), ("tf32x3", 2, 4), ("bf16x2", 1, 2), ("bf16x3", 2, 2)])
def test_table_bytes_follow_planes_and_element_size(mode, planes, es):
    r1 = _case(mode, 64, 1, 1, 1.0, 1000.0, 1000.0)
    r2 = _case(mode, 64, 2, 1, 1.0, 1000.0, 1000.0)
    assert math.isclose(r2["bytes"] - r1["bytes"], 2 * 64 * 64 * es * planes, rel_tol=1e-12)


def _bench_commands(text):
    """The bench.py argument lists of every `python bench.py ...` command in a text (shell
    line continuations joined, the `python bench.py` prefix and environment assignments
    dropped)."""
    import re
    import shlex

    text = re.sub(r"\\\n\s*", " ", text)
    out = []
    for line in text.splitlines():
        for m in re.finditer(r"python bench\.py([^|&;>]*)", line):
            out.append(shlex.split(m.group(1).replace("$v", "0"), comments=True))
    return out


def test_profile_and_readme_commands_parse():
    """Every bench command that a profile summary or the README gives is accepted by
    bench.py's own argument parser (so the recorded commands stay runnable)."""
    import glob
    import os

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = sorted(glob.glob(os.path.join(root, "profiles", "*.txt"))) + [os.path.join(root, "README.md")]
    seen = 0
    for f in files:
        for argv in _bench_commands(open(f).read()):
            bench.parse(argv)  # argparse exits (SystemExit) on an unknown flag or value
            seen += 1
    assert seen >= 10
