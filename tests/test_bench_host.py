"""Host-side helpers of bench.py's serving block (no GPU): the one-at-a-time queue that the
plain path's latencies come from, and the nearest-rank percentiles of p50 / p99."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fifo_queues_and_idles():
    # requests at t = 0, 1, 2 with 5 s of service each queue behind one another
    lat, end = bench.fifo([0.0, 1.0, 2.0], [5.0, 5.0, 5.0])
    assert lat == [5.0, 9.0, 13.0] and end == 15.0
    # a request that arrives after the server went idle waits for nothing
    lat, end = bench.fifo([0.0, 10.0], [2.0, 3.0])
    assert lat == [2.0, 3.0] and end == 13.0
    # latency is never below the request's own service time
    arr = [0.1 * i for i in range(50)]
    svc = [0.05 + 0.01 * (i % 7) for i in range(50)]
    lat, end = bench.fifo(arr, svc)
    assert all(l >= s - 1e-12 for l, s in zip(lat, svc))
    assert abs(end - max(a + l for a, l in zip(arr, lat))) < 1e-12


def test_percentiles_are_nearest_rank():
    vals = list(range(1, 101))
    assert bench._pct(vals, 0.5) == 51
    assert bench._pct(vals, 0.99) == 100
    assert bench._pct(vals, 0.0) == 1
    assert bench._pct([7.0], 0.99) == 7.0
    assert bench._pct([3, 1, 2], 0.5) == 2  # order of the input does not matter


def test_clock_rows_give_median_max_and_reasons():
    rows = "\n".join([
        "0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",
    ])
    c = bench.parse_clocks(rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.parse_clocks("0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active\n")
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.parse_clocks("") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_clock_sampler_stop_reads_its_process():
    class FakeProc:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            return "0, 2070, 2070, 1000, 0x0, Not Active, Not Active, Not Active, Not Active\n", ""

    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc, s.gpu = FakeProc(), 0
    assert s.stop()["sm_mhz"] == 2070.0
    s.proc = None
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
