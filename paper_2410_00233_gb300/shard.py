"""Host logic of the multi-GPU (data-parallel) path: one process per GPU, independent
problems per rank, no data-path collective.

Deblurs are independent (each request has its own PSF, image and noise), so the path shards
by request: rank r, step s takes the request ids ``request_ids(r, s, batch)``, disjoint
across ranks and steps.  The only collective is the timing reduction: the job's time is the
maximum over ranks, and its throughput counts the units of every rank (weak scaling: the
per-rank batch is fixed as the number of ranks grows).
"""
from __future__ import annotations

RANK_STRIDE = 100000  # request ids per rank (steps * batch must stay below this)


def request_ids(rank: int, step: int, batch: int) -> range:
    """Ids of the requests rank ``rank`` solves in step ``step`` (a batch of ``batch``)."""
    if not (0 <= rank and 0 <= step and 0 < batch and (step + 1) * batch <= RANK_STRIDE):
        raise ValueError(f"bad shard rank={rank} step={step} batch={batch}")
    first = rank * RANK_STRIDE + step * batch
    return range(first, first + batch)


def job_seconds(seconds_this_rank: float, dist=None, device=None) -> float:
    """Maximum over ranks of the per-rank time (all-reduce MAX; identity without a group)."""
    if dist is None:
        return float(seconds_this_rank)
    import torch

    t = torch.tensor([float(seconds_this_rank)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: units of all ranks over the job time."""
    return world * units_per_rank / seconds
