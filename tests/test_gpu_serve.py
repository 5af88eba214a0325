"""Serving loop: continuous batching, KP cache, admission by memory budget.

Requests submitted while others run join the running batch; each result must equal the
same request solved alone (kp_build with the same seed, then sb_solve with the same
settings), bit for bit: per-problem kernels with fixed-order reductions, and rounds that
only regroup whole outer steps.
"""
import time

import numpy as np
import pytest

from oracle import kpsb_oracle as O
from paper_2410_00233_gb300 import inputs as I
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _request(i, n=128):
    g = I.rng(7000 + i)
    psf = I.psf_gaussian_mixture(15, g)
    xt = I.image_piecewise_constant(n, g)
    bt = O.blur(psf, xt, I.BC_REFLEXIVE)
    b = bt + I.noise_vector(bt, 0.02, I.gaussian((n, n), g))
    return psf, b


@pytest.mark.parametrize("prec_name", ["P_TF32X2", "P_FP64"])
def test_served_results_equal_alone(prec_name):
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    prec = getattr(K, prec_name)
    iters = 4
    reqs = []
    for i in range(5):
        psf, b = _request(i if i != 4 else 1)  # request 4 repeats the PSF of request 1
        reqs.append(dict(psf=psf, b=b if i != 4 else b + 0.001, tv=K.ISO if i % 2 else K.ANISO,
                         key=1000 + (i if i != 4 else 1)))
    srv = K.Server(budget_bytes=8 << 30, max_active=4, round_steps=2)
    ids = []
    for r in reqs[:2]:
        ids.append(srv.submit(r["psf"], 128, K.BC_REFLEXIVE, 6, r["b"], 1.0, 0.1, r["tv"], iters,
                              prec=prec, psf_key=r["key"]))
    time.sleep(0.3)  # the first two are running when the others arrive
    for r in reqs[2:]:
        ids.append(srv.submit(r["psf"], 128, K.BC_REFLEXIVE, 6, r["b"], 1.0, 0.1, r["tv"], iters,
                              prec=prec, psf_key=r["key"]))
    outs = [srv.poll(i, timeout_us=30_000_000) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == 5 and st["failed"] == 0
    assert st["cache_hits"] >= 1  # request 4 reused the factors of request 1
    assert st["peak_bytes"] <= 8 << 30
    for r, (x, stats, lat) in zip(reqs, outs):
        kp = K.kp_build(r["psf"], 128, K.BC_REFLEXIVE, 6, K.EGKB, seed=r["key"])
        xa, sa = K.sb_solve(kp, r["b"], 1.0, 0.1, r["tv"], iters, prec=prec)
        assert np.array_equal(x, xa)
        assert stats.l_end == sa.l_end == iters and stats.iota_total == sa.iota_total
        assert lat > 0


def test_server_refuses_what_never_fits_and_admits_within_budget():
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    psf, b = _request(9)
    tiny = K.Server(budget_bytes=1 << 20, max_active=2)
    rid = tiny.submit(psf, 128, K.BC_REFLEXIVE, 4, b, 1.0, 0.1, K.ANISO, 2, prec=K.P_FP32)
    with pytest.raises(K.KpsbError) as e:
        tiny.poll(rid, timeout_us=30_000_000)
    assert e.value.code == -7  # EBUSY
    tiny.close()
    # a budget for about two requests at a time (state ~2.2 MB each, factors 0.5 MB) still
    # completes six, never exceeding it
    srv = K.Server(budget_bytes=6 << 20, max_active=8, round_steps=1)
    ids = [srv.submit(psf, 128, K.BC_REFLEXIVE, 4, b, 1.0, 0.1, K.ANISO, 2, prec=K.P_FP32, psf_key=5)
           for _ in range(6)]
    res = [srv.poll(i, timeout_us=30_000_000) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == 6 and st["peak_bytes"] <= 6 << 20
    for x, _, _ in res[1:]:
        assert np.array_equal(x, res[0][0])


@pytest.mark.parametrize("n,P", [(128, 200), (256, 40)])
def test_same_bits_alone_in_a_large_batch_and_served(n, P, monkeypatch):
    """One request solved three ways gives the same bits: alone, inside a batch of P other
    problems (cut into concurrent parts), and in a server round with other requests.  The lone
    solve is forced onto the two-stage apply kernel while the batch runs whatever the tuner
    picks for its size (the resident or tiled fused kernel): every apply variant issues the
    same MMAs for each output element, and every vector kernel treats a problem on its own with
    fixed-order reductions."""
    need_gpu()
    from paper_2410_00233_gb300 import kpsb as K

    g = I.rng(4242 + n)
    jobs = []
    for p in range(P):
        k = 3 + p % 9
        kp = K.kp_from_factors((g.standard_normal((k, n, n)) / n).astype(np.float32),
                               (g.standard_normal((k, n, n)) / n).astype(np.float32),
                               np.sort(g.random(k))[::-1] + 0.1)
        jobs.append(dict(kp=kp, b=g.standard_normal((n, n)), mu=1.0, lam=0.1,
                         tv=K.ISO if p % 2 else K.ANISO, iters=2))
    outs, stats = K.sb_solve_batched(jobs, prec=K.P_TF32X2)
    psf, b = _request(31, n)
    kp_t = K.kp_build(psf, n, K.BC_REFLEXIVE, 6, K.EGKB, seed=777)
    monkeypatch.setenv("KPSB_TC_VARIANT", "0")  # two-stage kernels for the lone solve
    x_alone, st_alone = K.sb_solve(kp_t, b, 1.0, 0.1, K.ISO, 2, prec=K.P_TF32X2)
    monkeypatch.delenv("KPSB_TC_VARIANT")
    # the same request inside a batch with the P others
    outs2, stats2 = K.sb_solve_batched(jobs[:P // 2] + [dict(kp=kp_t, b=b, mu=1.0, lam=0.1, tv=K.ISO, iters=2)]
                                       + jobs[P // 2:], prec=K.P_TF32X2)
    assert np.array_equal(outs2[P // 2], x_alone) and stats2[P // 2].iota_total == st_alone.iota_total
    for a, c in zip(outs[:3] + outs[-3:], outs2[:3] + outs2[-3:]):
        assert np.array_equal(a, c)
    # and served, with other requests in the same rounds
    srv = K.Server(budget_bytes=8 << 30, max_active=16, round_steps=1)
    ids = []
    for i in range(6):
        psf_i, b_i = _request(40 + i, n)
        ids.append(srv.submit(psf_i, n, K.BC_REFLEXIVE, 6, b_i, 1.0, 0.1, K.ANISO, 2, prec=K.P_TF32X2,
                              psf_key=500 + i))
    tid = srv.submit(psf, n, K.BC_REFLEXIVE, 6, b, 1.0, 0.1, K.ISO, 2, prec=K.P_TF32X2, psf_key=777)
    x_srv, st_srv, _ = srv.poll(tid, timeout_us=60_000_000)
    for i in ids:
        srv.poll(i, timeout_us=60_000_000)
    srv.close()
    assert np.array_equal(x_srv, x_alone) and st_srv.iota_total == st_alone.iota_total
