"""Replica bookkeeping for runs on several GPUs.

The apply has no exchange step between suspensions, so several GPUs only
run independent replicas: every rank owns a disjoint share of the units (whole
suspensions of a batch, or whole requests) and the job's time is the maximum
over the ranks.  Nothing here touches device data.
"""
from __future__ import annotations


def shard(n_units: int, rank: int, world: int, costs=None):
    """Indices of the units owned by `rank`.  Without costs: round robin.
    With costs: longest-processing-time first onto the least loaded rank, so
    that uneven suspensions balance; every rank computes the same split."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    if costs is None:
        return list(range(rank, n_units, world))
    order = sorted(range(n_units), key=lambda k: (-costs[k], k))
    load = [0.0] * world
    owner = [0] * n_units
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += costs[k]
    return [k for k in range(n_units) if owner[k] == rank]


def max_over_ranks(value: float, world: int) -> float:
    """Maximum of a host float over all ranks (gloo or nccl process group)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
