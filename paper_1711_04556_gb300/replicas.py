"""Independent searches spread over ranks, one GPU per rank.

Instances are independent, so N GPUs run N replicas of the search path,
each on its own part of the instances.  Two ways to split:

* `shard`: every rank takes its own consecutive seeds (weak scaling: the
  work per GPU stays fixed as N grows);
* `lpt_partition`: one fixed batch split by estimated cost, longest first,
  each instance to the least-loaded rank (strong scaling), with
  `gather_results` bringing every rank's results back to rank 0 in the
  batch's order.

There is no data-path collective: the only cross-rank traffic is a barrier,
the reduction of timings and counts (max of the device times, sum of the
evaluated schedules), and the gather of results on the host.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard(family: str, per_rank: int, rank: int) -> List:
    """The instances rank `rank` solves: `per_rank` consecutive seeds."""
    from . import instances
    return instances.config_batch(family, per_rank, first=rank * per_rank)


def potential_moves(n: int, delta: int) -> int:
    """Swaps (u, v) of the reduced neighbourhood: 1 <= u < v <= N-2,
    v - u <= delta (Sec. 4.3), N = n activities with the dummies."""
    return sum(min(delta, n - 2 - u) for u in range(1, n - 2))


def estimated_cost(inst, iterations: int, delta: int = 0) -> int:
    """Decode work of one search, up to a constant: N activities placed for
    every potential move of every iteration.  delta = 0 takes the swap
    distance the library uses for the instance's size."""
    from . import instances
    d = delta or instances.search_params(inst.n - 2)[0]
    d = max(1, min(d, inst.n - 3))
    return inst.n * potential_moves(inst.n, d) * iterations


def lpt_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest processing time first: instances by falling cost (ties: lower
    index first), each to the rank with the least load so far (ties: lower
    rank).  Returns each rank's indices in ascending order; the same on every
    rank, since it depends on the costs only."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_results(dist, results: Sequence, indices: Sequence[int], total: int, world: int, rank: int):
    """Rank 0 receives every rank's (index, result) pairs and returns the
    results of the whole batch in its order; the other ranks return None."""
    if world <= 1:
        out = [None] * total
        for i, r in zip(indices, results):
            out[i] = r
        return out
    payload = list(zip(indices, results))
    recv = [None] * world if rank == 0 else None
    dist.gather_object(payload, recv, dst=0)
    if rank != 0:
        return None
    out = [None] * total
    for part in recv:
        for i, r in part:
            if out[i] is not None:
                raise RuntimeError(f"instance {i} solved twice")
            out[i] = r
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"instances without a result: {missing[:8]}")
    return out


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
