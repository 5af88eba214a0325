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
