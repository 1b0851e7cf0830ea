"""Independent searches spread over ranks, one GPU per rank.

Instances are independent, so N GPUs run N replicas of the search path,
each on its own shard of instances (weak scaling).  There is no data-path
collective: the only cross-rank traffic is a barrier and the reduction of
timings and counts (max of the device times, sum of the evaluated
schedules).
"""
from __future__ import annotations

from typing import List, Tuple


def shard(family: str, per_rank: int, rank: int) -> List:
    """The instances rank `rank` solves: `per_rank` consecutive seeds."""
    from . import instances
    return instances.config_batch(family, per_rank, first=rank * per_rank)


def reduce_timing(dist, device, seconds: float, schedules: float, world: int) -> Tuple[float, float]:
    """(max of `seconds`, sum of `schedules`) over the ranks of `dist`."""
    if world <= 1:
        return seconds, schedules
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    e = torch.tensor([schedules], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())
