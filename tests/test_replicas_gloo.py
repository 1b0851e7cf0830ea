"""The multi-rank replica path on CPU: two gloo ranks.

Each rank takes its own shard of instances (no instance solved twice, the
same shard every run) and the timing reduction returns the slowest rank's
time and the total count, as the benchmark reports for N GPUs.  With one
batch split by cost, ranks that search their shares (with the oracle, on
the CPU) and gather on rank 0 give the results of one process.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1711_04556_gb300 import replicas
    insts = replicas.shard("j30_batch", 6, rank)
    digests = [x.digest() for x in insts]
    t, e = replicas.reduce_timing(dist, "cpu", 1.0 + rank, 10.0 * (rank + 1), world)
    gathered = [None] * world
    dist.all_gather_object(gathered, digests)
    out[rank] = (t, e, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, e, gathered = out[r]
        assert t == 2.0 and e == 30.0
        assert not set(gathered[0]) & set(gathered[1])          # disjoint shards
    from paper_1711_04556_gb300 import replicas
    assert [x.digest() for x in replicas.shard("j30_batch", 6, 1)] == out[0][2][1]


# ------------------------------------------- one batch split by LPT over ranks
def _lpt_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1711_04556_gb300 import instances, replicas
    batch = instances.config_batch("mixed_batch", 40)
    costs = [replicas.estimated_cost(x, 1000) for x in batch]
    parts = replicas.lpt_partition(costs, world)
    mine = parts[rank]
    # a stand-in for the search: what a rank reports about each instance
    results = [{"digest": batch[i].digest(), "rank": rank} for i in mine]
    got = replicas.gather_results(dist, results, mine, len(batch), world, rank)
    out[rank] = (parts, got)
    dist.barrier()
    dist.destroy_process_group()


def test_lpt_split_and_gather_over_two_gloo_ranks():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_lpt_rank, args=(world, port, out), nprocs=world, join=True)
    from paper_1711_04556_gb300 import instances
    batch = instances.config_batch("mixed_batch", 40)
    parts0, got = out[0]
    assert out[1][0] == parts0 and out[1][1] is None             # same split everywhere; rank 0 gathers
    assert sorted(parts0[0] + parts0[1]) == list(range(40))
    assert [g["digest"] for g in got] == [x.digest() for x in batch]
    assert all(g["rank"] == (0 if i in parts0[0] else 1) for i, g in enumerate(got))


def test_lpt_partition_bounds():
    """Greedy list scheduling keeps every rank within total/m + the largest
    cost, and LPT within Graham's (4/3 - 1/(3m)) of the optimum (brute force
    on small cases)."""
    import itertools
    import random
    from paper_1711_04556_gb300 import replicas
    rnd = random.Random(5)
    for trial in range(300):
        m = rnd.randint(1, 4)
        costs = [rnd.randint(1, 50) for _ in range(rnd.randint(0, 9))]
        parts = replicas.lpt_partition(costs, m)
        assert len(parts) == m and sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        if costs:
            assert max(loads) <= sum(costs) / m + max(costs)
            opt = min(max(sum(c for c, r in zip(costs, a) if r == q) for q in range(m))
                      for a in itertools.product(range(m), repeat=len(costs)))
            assert max(loads) <= (4 / 3 - 1 / (3 * m)) * opt + 1e-9
        assert replicas.lpt_partition(costs, m) == parts


def test_potential_moves_is_the_neighbourhood_size(oracle):
    """With no precedence between the non-dummy activities every swap is
    feasible, so one iteration decodes exactly the potential moves."""
    import numpy as np
    from paper_1711_04556_gb300 import replicas
    from paper_1711_04556_gb300.instances import Instance
    for n_act, delta in ((5, 2), (12, 4), (12, 20), (30, 20)):
        n = n_act + 2
        succ = [list(range(1, n - 1))] + [[n - 1] for _ in range(n_act)] + [[]]
        off = np.r_[0, np.cumsum([len(s) for s in succ])].astype(np.int32)
        inst = Instance(n, 1, np.r_[0, np.ones(n_act), 0].astype(np.int32), np.array([2], np.int32),
                        np.r_[0, np.ones(n_act), 0].astype(np.int32), off,
                        np.array([x for s in succ for x in s], np.int32))
        r = oracle.tabu_search(inst, 1, delta, 5, 1, 0)
        brute = sum(1 for u in range(1, n - 2) for v in range(u + 1, n - 1) if v - u <= delta)
        assert r["evaluated"] == brute == replicas.potential_moves(n, delta)


# ------------------- the strong-scaling path with real per-rank search results
def _lpt_search_rank(rank, world, port, out):
    """Each rank searches its longest-processing-time share of one batch --
    with the oracle, the CPU stand-in for a rank's GPU -- and rank 0 gathers
    the results in batch order, as bench.py --shard lpt does."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1711_04556_gb300 import instances, replicas
    batch = instances.config_batch("mixed_batch", 12)
    parts = replicas.lpt_partition([replicas.estimated_cost(x, 40) for x in batch], world)
    mine = parts[rank]
    params = [(40,) + instances.search_params(batch[i].n - 2) + (O.AUTO, 1) for i in mine]
    found = O.tabu_search_batch([batch[i] for i in mine], params, 2)
    results = [{"best_cmax": r["best_cmax"], "evaluated": r["evaluated"], "work": r["work"],
                "best_W": np.asarray(r["best_W"]).tolist(), "rank": rank} for r in found]
    got = replicas.gather_results(dist, results, mine, len(batch), world, rank)
    out[rank] = (parts, got)
    dist.barrier()
    dist.destroy_process_group()


def test_lpt_shards_searched_and_gathered_equal_one_process(oracle):
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_lpt_search_rank, args=(world, port, out), nprocs=world, join=True)
    from paper_1711_04556_gb300 import instances
    batch = instances.config_batch("mixed_batch", 12)
    parts, got = out[0]
    assert out[1][1] is None and len(got) == len(batch)
    assert {g["rank"] for g in got} == {0, 1}                     # both ranks did work
    params = [(40,) + instances.search_params(x.n - 2) + (oracle.AUTO, 1) for x in batch]
    for g, r in zip(got, oracle.tabu_search_batch(batch, params, 2)):
        assert g["best_cmax"] == r["best_cmax"] and g["evaluated"] == r["evaluated"] and g["work"] == r["work"]
        assert g["best_W"] == np.asarray(r["best_W"]).tolist()
