"""The data-parallel host logic with two ranks on CPU (gloo): disjoint request ids per rank
and step, and the job time as the maximum over ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, steps, batch, q):
    import torch.distributed as dist

    from paper_2410_00233_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = [list(shard.request_ids(rank, s, batch)) for s in range(steps)]
        gathered = [None] * world
        dist.all_gather_object(gathered, ids)
        t = shard.job_seconds(1.0 + rank, dist)  # rank 1 is the slow one
        q.put((rank, gathered, t, shard.throughput(batch * steps, world, t)))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_are_disjoint_and_time_is_the_max():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, steps, batch = _free_port(), 3, 5
    procs = [ctx.Process(target=_worker, args=(r, 2, port, steps, batch, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t, value in res:
        assert t == 2.0 and value == 2 * batch * steps / 2.0
        flat = [i for r in gathered for step in r for i in step]
        assert len(flat) == len(set(flat)) == 2 * steps * batch  # disjoint across ranks and steps
    assert res[0][1] == res[1][1]


def test_request_ids_reject_overflowing_shards():
    from paper_2410_00233_gb300 import shard

    with pytest.raises(ValueError):
        shard.request_ids(0, shard.RANK_STRIDE, 1)
    assert list(shard.request_ids(1, 2, 3)) == [shard.RANK_STRIDE + 6, shard.RANK_STRIDE + 7, shard.RANK_STRIDE + 8]
