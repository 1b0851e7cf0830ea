"""Sliced launches (rcpsp_params.slices).

A launch class with more searches than its CTAs hold at once runs every
search in slices of ceil(iterations / slices) iterations; between slices the
search's state waits in device memory, and the next slice may run on another
CTA.  Slicing changes only the order in which the GPU works, never a
result: every test compares the sliced searches with the same searches run
unsliced (best list, schedule, makespan, iteration and neighbour counts, the
paper's work counter, the performed-work counters and the trace) and with
the oracle.  Forced slice counts on small batches make CTAs wait for a slice
that another CTA is still running.
"""
import os
import shutil

import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R

pytestmark = pytest.mark.gpu

NPROC = os.cpu_count() or 1
KEYS = ("best_cmax", "iterations", "evaluated", "work", "mode", "cp", "status", "placements", "steps_done",
        "update_units", "succ_pushes", "kept_words")
HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(os.path.dirname(HERE), "paper_1711_04556_gb300", "tune_shapes.tsv")


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


def same_as_oracle(g, r):
    assert g["status"] == 0
    for k in ("best_cmax", "iterations", "evaluated", "work", "mode", "cp"):
        assert g[k] == r[k], k
    assert g["best_W"].tolist() == r["best_W"].tolist()
    assert g["best_S"].tolist() == r["best_S"].tolist()


def batch():
    return (I.config_batch("j30_batch", 40, first=60) + I.config_batch("j120_batch", 4, first=10)
            + [x for x in I.config_batch("mixed_batch", 40) if x.n <= 122][:6])


@pytest.mark.parametrize("slices", [3, 7])
def test_forced_slices_equal_unsliced_and_oracle(solver, oracle, slices):
    insts = batch()
    ids = solver.load(insts)
    kw = dict(iterations=70, delta=0, tabu_len=0, mode=R.EVAL_AUTO, trace=True)
    solver.search(ids, slices=1, **kw)
    ref = solver.results(ids)
    ref_tr = [solver.trace(i, 70).tolist() for i in ids]
    assert all(c["slices"] == 1 for c in solver.last_launches())
    solver.search(ids, slices=slices, **kw)
    got = solver.results(ids)
    assert all(c["slices"] == slices for c in solver.last_launches())
    for k, (a, b) in enumerate(zip(got, ref)):
        same(a, b)
        assert solver.trace(ids[k], 70).tolist() == ref_tr[k]
    params = [(70,) + I.search_params(x.n - 2) + (oracle.AUTO, 1) for x in insts]
    for g, r in zip(got, oracle.tabu_search_batch(insts, params, NPROC)):
        same_as_oracle(g, r)
    solver.free(ids)


@pytest.mark.parametrize("csize", [2, 4])
def test_slices_on_clusters(solver, oracle, csize):
    insts = I.config_batch("j120_batch", 6, first=30)
    ids = solver.load(insts)
    kw = dict(iterations=40, delta=60, tabu_len=800, mode=R.EVAL_AUTO, cluster_size=csize)
    solver.search(ids, slices=1, **kw)
    ref = solver.results(ids)
    solver.search(ids, slices=5, **kw)
    for a, b in zip(solver.results(ids), ref):
        same(a, b)
    params = [(40, 60, 800, oracle.AUTO, 1)] * len(insts)
    for g, r in zip(ref, oracle.tabu_search_batch(insts, params, NPROC)):
        same_as_oracle(g, r)
    solver.free(ids)


def test_slices_with_checkpoint_and_resume(solver):
    """A sliced call that keeps its state, resumed by another sliced call,
    ends as one unsliced call of both lengths."""
    insts = batch()
    ids = solver.load(insts)
    kw = dict(delta=0, tabu_len=0, mode=R.EVAL_AUTO)
    solver.search(ids, iterations=60, slices=1, **kw)
    ref = solver.results(ids)
    solver.search(ids, iterations=23, checkpoint=True, slices=4, **kw)
    solver.search(ids, iterations=37, resume=True, checkpoint=True, slices=6, **kw)
    for a, b in zip(solver.results(ids), ref):
        for k in ("best_cmax", "iterations", "evaluated", "work", "mode", "cp", "status"):
            assert a[k] == b[k], k
        assert a["best_W"].tolist() == b["best_W"].tolist()
        assert a["best_S"].tolist() == b["best_S"].tolist()
    solver.free(ids)


def test_graph_replay_of_a_sliced_launch(solver):
    import torch
    st = torch.cuda.Stream()
    insts = I.config_batch("j30_batch", 64, first=300)
    ids = solver.load(insts)
    kw = dict(iterations=120, delta=20, tabu_len=60, mode=R.EVAL_AUTO, stream=st)
    solver.search(ids, slices=1, **kw)
    ref = solver.results(ids)
    for _ in range(3):   # the replays re-zero the slice counters
        solver.search(ids, slices=5, use_graph=True, **kw)
        for a, b in zip(solver.results(ids), ref):
            same(a, b)
    solver.free(ids)


def test_automatic_slices_on_the_j30_batch(solver, oracle, tmp_path, monkeypatch):
    """480 x 1000 iterations at the measured shapes: the main class has more
    searches than CTAs, so it is sliced; the results are the oracle's."""
    table = tmp_path / "shapes.tsv"
    shutil.copyfile(TABLE, table)
    monkeypatch.setenv("RCPSP_TUNE_CACHE", str(table))
    with R.Solver(0) as s:
        insts = I.config_batch("j30_batch")
        ids = s.load(insts)
        s.search(ids, iterations=1000, delta=20, tabu_len=60, mode=R.EVAL_AUTO)
        got = s.results(ids)
        plan = s.last_launches()
        assert any(c["slices"] > 1 and c["searches"] > c["ctas"] for c in plan), plan
        assert all(c["slices"] == 1 for c in plan if c["searches"] <= c["ctas"] // c["cluster_size"])
        s.search(ids, iterations=1000, delta=20, tabu_len=60, mode=R.EVAL_AUTO, slices=1)
        for a, b in zip(got, s.results(ids)):
            same(a, b)
    ref = oracle.tabu_search_batch(insts, [(1000, 20, 60, 0, 1)] * len(insts), NPROC)
    for g, r in zip(got, ref):
        same_as_oracle(g, r)


def test_slice_count_limits(solver):
    ids = solver.load(I.config_batch("j30_batch", 2))
    for bad in (-1, 65):
        p = R.Params(10, 20, 60, 0, 1, 0, 0, 0, 0, 0, 0, 0, bad)
        assert solver.lib.rcpsp_tabu_search(solver.ctx, R._ptr(ids), len(ids), R.C.byref(p), None) == R.E_INVALID_ARG
    solver.search(ids, iterations=3, delta=20, tabu_len=60, slices=64)   # more slices than iterations
    assert all(r["status"] == 0 and r["iterations"] <= 3 for r in solver.results(ids))
    solver.free(ids)
