"""Checkpoint and resume of searches (rcpsp_params.checkpoint / resume,
rcpsp_get_state / rcpsp_set_state).

The search loop draws no random numbers, so a search kept after k1
iterations and resumed for k2 more must end exactly as one search of k1 + k2
iterations: the same best list, schedule and makespan, and the same
iteration, neighbour and work counts; the trace of the resumed call is the
tail of the uninterrupted trace.  Also across contexts (state copied out
and back in), on clusters, with graph replays, and the error cases.
"""
import os

import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R

pytestmark = pytest.mark.gpu

NPROC = os.cpu_count() or 1
KEYS = ("best_cmax", "iterations", "evaluated", "work", "mode", "cp", "status")


@pytest.fixture(scope="module")
def solver():
    from paper_1711_04556_gb300 import build as B
    B.build()
    s = R.Solver(0)
    yield s
    s.close()


def same(a, b):
    for k in KEYS:
        assert a[k] == b[k], k
    assert a["best_W"].tolist() == b["best_W"].tolist()
    assert a["best_S"].tolist() == b["best_S"].tolist()


def batch():
    return (I.config_batch("j30_batch", 40, first=60) + I.config_batch("j120_batch", 4, first=10)
            + [x for x in I.config_batch("mixed_batch", 30) if x.n <= 92][:4])


@pytest.mark.parametrize("mode", [R.EVAL_AUTO, R.EVAL_TIME, R.EVAL_CAPACITY])
def test_resumed_search_equals_uninterrupted(solver, oracle, mode):
    insts = batch()
    ids = solver.load(insts)
    kw = dict(delta=0, tabu_len=0, mode=mode, stop_at_cp=True)
    solver.search(ids, iterations=70, trace=True, **kw)
    ref = solver.results(ids)
    ref_tr = [solver.trace(i, 70) for i in ids]
    solver.search(ids, iterations=25, checkpoint=True, **kw)
    solver.search(ids, iterations=30, checkpoint=True, resume=True, **kw)
    solver.search(ids, iterations=15, resume=True, trace=True, **kw)
    got = solver.results(ids)
    for k, (a, b) in enumerate(zip(got, ref)):
        same(a, b)
        done = b["iterations"]
        tail = ref_tr[k][55:done] if done > 55 else ref_tr[k][:0]
        assert solver.trace(ids[k], 15)[:len(tail)].tolist() == tail.tolist()
    solver.free(ids)
    # and the uninterrupted search is the oracle's
    params = [(70,) + I.search_params(x.n - 2) + (mode, 1) for x in insts]
    for a, r in zip(got, oracle.tabu_search_batch(insts, params, NPROC)):
        assert a["best_cmax"] == r["best_cmax"] and a["evaluated"] == r["evaluated"]
        assert a["best_W"].tolist() == r["best_W"].tolist()


def test_state_moves_between_contexts(solver):
    insts = I.config_batch("j30_batch", 16, first=5)
    ids = solver.load(insts)
    solver.search(ids, iterations=90, delta=20, tabu_len=60)
    ref = solver.results(ids)
    solver.search(ids, iterations=40, delta=20, tabu_len=60, checkpoint=True)
    states = [solver.get_state(i) for i in ids]
    solver.free(ids)
    with R.Solver(0) as other:
        ids2 = other.load(insts)
        for i, st in zip(ids2, states):
            other.set_state(i, st)
        other.search(ids2, iterations=50, delta=20, tabu_len=60, resume=True)
        for a, b in zip(other.results(ids2), ref):
            same(a, b)


@pytest.mark.parametrize("csize", [2, 4])
def test_resume_on_clusters(solver, csize):
    insts = I.config_batch("j120_batch", 6, first=20)
    ids = solver.load(insts)
    solver.search(ids, iterations=24, delta=60, tabu_len=800)
    ref = solver.results(ids)
    solver.search(ids, iterations=10, delta=60, tabu_len=800, checkpoint=True, cluster_size=csize)
    solver.search(ids, iterations=14, delta=60, tabu_len=800, resume=True, cluster_size=1)
    for a, b in zip(solver.results(ids), ref):
        same(a, b)
    solver.search(ids, iterations=10, delta=60, tabu_len=800, checkpoint=True, cluster_size=1)
    solver.search(ids, iterations=14, delta=60, tabu_len=800, resume=True, cluster_size=csize)
    for a, b in zip(solver.results(ids), ref):
        same(a, b)
    solver.free(ids)


def test_time_slices_by_graph_replay(solver):
    """The same resumed launch replayed from a CUDA graph advances the
    searches slice by slice."""
    import torch
    st = torch.cuda.Stream()
    insts = I.config_batch("j30_batch", 48, first=100)
    ids = solver.load(insts)
    solver.search(ids, iterations=100, delta=20, tabu_len=60, stream=st)
    ref = solver.results(ids)
    solver.search(ids, iterations=0, delta=20, tabu_len=60, checkpoint=True, stream=st)
    for _ in range(4):
        solver.search(ids, iterations=25, delta=20, tabu_len=60, checkpoint=True, resume=True, use_graph=True,
                      stream=st)
    for a, b in zip(solver.results(ids), ref):
        same(a, b)
    solver.free(ids)


def test_checkpoint_errors(solver):
    x = I.config_batch("j30_batch", 2)
    ids = solver.load(x)
    with pytest.raises(R.RcpspError) as e:                     # nothing kept yet
        solver.search(ids, iterations=5, resume=True)
    assert e.value.code == -1
    with pytest.raises(R.RcpspError) as e:
        solver.get_state(ids[0])
    assert e.value.code == -1
    solver.search(ids, iterations=5, delta=20, tabu_len=60, checkpoint=True)
    with pytest.raises(R.RcpspError) as e:                     # kept with other parameters
        solver.search(ids, iterations=5, delta=10, tabu_len=60, resume=True)
    assert e.value.code == -1
    st = solver.get_state(ids[0])
    other = I.config_batch("j120_batch", 1)
    oid = solver.load(other)
    with pytest.raises(R.RcpspError) as e:                     # another instance's state
        solver.set_state(oid[0], st)
    assert e.value.code == -1
    bad = bytearray(st)
    bad[0] ^= 1
    with pytest.raises(R.RcpspError) as e:
        solver.set_state(ids[1], bytes(bad))
    assert e.value.code == -1
    import ctypes as C
    arr = R._i32(ids)
    for flags in ((1, 0), (0, 1)):                             # not on the no-allocation path
        p = R.Params(5, 20, 60, 0, 1, 0, 0, 0, 0, 0, *flags)
        assert solver.lib.rcpsp_tabu_search_noalloc(solver.ctx, R._ptr(arr), len(arr), C.byref(p), None) == -1
    solver.free(ids)
    solver.free(oid)
