"""The multi-rank replica path on CPU: two gloo ranks.

Each rank takes its own shard of instances (no instance solved twice, the
same shard every run) and the timing reduction returns the slowest rank's
time and the total count, as the benchmark reports for N GPUs.
"""
import os
import socket

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
