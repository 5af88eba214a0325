"""kp_build's argument checks (include/kpsb.h) on random arguments, no GPU: every argument
set the header rules out returns KPSB_EINVAL before any device work, and every other set
returns a defined status (without a GPU, the first device allocation fails) -- never a crash.

The rules: 2 <= n <= KPSB_MAX_N; PSF sides in [1, 1024]; boundary 0 or 1, with the reflexive
overhang s/2 and s - 1 - s/2 at most n on both sides; method EGKB or RSVD; rank_or_tol > 0
and finite, a fixed rank k = floor(rank_or_tol) in [1, 64] when >= 1, automatic rank (< 1)
only with EGKB and capped at 30 terms; k_p = k + p <= 64 with the default p = max(2, ceil(k/4)).
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2410_00233_gb300 import kpsb as K

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


def _valid(s0, s1, n, bc, r, method):
    if not (2 <= n <= 16384 and 1 <= s0 <= 1024 and 1 <= s1 <= 1024 and bc in (0, 1) and method in (0, 1)):
        return False
    if bc == 1 and not (s0 // 2 <= n and s1 // 2 <= n and s0 - 1 - s0 // 2 <= n and s1 - 1 - s1 // 2 <= n):
        return False
    if not (r > 0 and math.isfinite(r)):
        return False
    if r >= 1.0:
        k = int(r)
        return 1 <= k <= 64 and k + max(2, (k + 3) // 4) <= 64
    return method == 0  # automatic rank: k_cap 30, p 8, k_p 38


@hyp.settings(max_examples=300, deadline=None, derandomize=True)
@hyp.given(s0=st.integers(-2, 1030), s1=st.integers(-2, 1030), n=st.sampled_from([-1, 0, 1, 2, 3, 8, 100, 16384, 16385]),
           bc=st.integers(-1, 2), r=st.one_of(st.floats(-2, 80), st.sampled_from([0.0, math.nan, math.inf, 51.0, 52.0])),
           method=st.integers(-1, 2))
def test_kp_build_rejects_exactly_what_the_header_rules_out(s0, s1, n, bc, r, method):
    L = K.lib()
    ns0, ns1 = max(s0, 1), max(s1, 1)
    if ns0 * ns1 > 1 << 16:  # keep the host PSF small; the sides still reach the limits below
        ns0, ns1 = min(ns0, 256), min(ns1, 256)
        s0, s1 = ns0 if s0 > 0 else s0, ns1 if s1 > 0 else s1
    psf = np.full((ns0, ns1), 1.0 / (ns0 * ns1), order="F")
    out = ctypes.c_void_p()
    rc = L.kp_build(psf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), s0, s1, n, bc, float(r), method, None,
                    ctypes.byref(out))
    assert rc in K.STATUS
    if not _valid(s0, s1, n, bc, r, method):
        assert rc == -1, (s0, s1, n, bc, r, method, rc, K.last_error())
    elif rc == 0:
        K.KP(out.value, n).close()  # only on a machine with a GPU
    else:
        assert rc != -1, (s0, s1, n, bc, r, method, K.last_error())
