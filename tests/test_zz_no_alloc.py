"""The search without device allocation (rcpsp_tabu_search_noalloc).

Some callers cannot allocate device memory when they search -- a serving
process whose device memory belongs to another allocator with a fixed
budget, or a host thread that may not wait on the device synchronisation
that cudaMalloc / cudaFree can imply.  For them the library offers a
variant of the search launch whose plan and work-queue counter live in a
fixed array inside the library.  Through the C interface it must give the
same results as rcpsp_tabu_search and as the CPU reference, on two calls in
a row (the second call finds the array holding the first call's plan and
counter).

This file is named so that pytest collects it last.
"""
import os

import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R

pytestmark = pytest.mark.gpu

KEYS = ("best_cmax", "iterations", "evaluated", "work", "mode", "cp", "status")
NPROC = os.cpu_count() or 1
# (1 MiB - 256 bytes) / 128-byte plan entries
MAX_ITEMS = ((1 << 20) - 256) // 128


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


def test_noalloc_matches_allocating_search_and_oracle_twice(solver, oracle):
    import torch
    # j30 and j120 searches plus uneven sizes up to N = 302 with M = 8
    mixed = [x for x in I.config_batch("mixed_batch", 64) if x.n == 302 and x.m == 8][:2]
    assert len(mixed) == 2
    insts = I.config_batch("j30_batch", 64, first=200) + I.config_batch("j120_batch", 4) + mixed
    ids = solver.load(insts)
    st = torch.cuda.Stream()
    kw = dict(iterations=120, delta=0, tabu_len=0, mode=R.EVAL_AUTO)
    solver.search(ids, stream=st, **kw)
    ref = solver.results(ids)
    params = [(120, *I.search_params(x.n - 2), oracle.AUTO, 1) for x in insts]
    for g, r in zip(ref, oracle.tabu_search_batch(insts, params, NPROC)):
        same_as_oracle(g, r)
    for _ in range(2):
        solver.search_noalloc(ids, stream=st, **kw)
        got = solver.results(ids)
        for a, b in zip(got, ref):
            same(a, b)
    # a different batch afterwards reuses the same array
    sub = ids[::3]
    solver.search(sub, stream=st, iterations=40, delta=20, tabu_len=60, mode=R.EVAL_CAPACITY)
    ref2 = solver.results(sub)
    solver.search_noalloc(sub, stream=st, iterations=40, delta=20, tabu_len=60, mode=R.EVAL_CAPACITY)
    for a, b in zip(solver.results(sub), ref2):
        same(a, b)
    solver.free(ids)


def test_noalloc_limits(solver, oracle):
    inst = I.config_batch("j30_single")[0]
    ids = solver.load([inst])
    params = R.Params(0, 0, 0, 0, 1, 0, 0, 0, 0)     # iterations = 0: only the initial list
    too_many = np.full(MAX_ITEMS + 1, ids[0], np.int32)
    rc = solver.lib.rcpsp_tabu_search_noalloc(solver.ctx, R._ptr(too_many), too_many.size, R.C.byref(params), None)
    assert rc == R.E_TOO_LARGE
    # exactly as many as the array holds is accepted (every entry the same search)
    full = np.full(MAX_ITEMS, ids[0], np.int32)
    rc = solver.lib.rcpsp_tabu_search_noalloc(solver.ctx, R._ptr(full), full.size, R.C.byref(params), None)
    assert rc == 0
    got = solver.results(ids)[0]
    ref = oracle.tabu_search(inst, 0, 20, 60, oracle.AUTO, 1)
    same_as_oracle(got, ref)
    traced = R.Params(10, 0, 0, 0, 1, 0, 0, 1, 0)    # record_trace = 1
    one = np.asarray(ids, np.int32)
    rc = solver.lib.rcpsp_tabu_search_noalloc(solver.ctx, R._ptr(one), 1, R.C.byref(traced), None)
    assert rc == R.E_INVALID_ARG
    for cs in (2, 3, -1, 16):                         # one CTA per search only
        clustered = R.Params(10, 0, 0, 0, 1, 0, 0, 0, 0, cs)
        rc = solver.lib.rcpsp_tabu_search_noalloc(solver.ctx, R._ptr(one), 1, R.C.byref(clustered), None)
        assert rc == R.E_INVALID_ARG
    solver.free(ids)


def test_noalloc_then_larger_search_on_another_context(solver, oracle):
    """The no-allocation call must not lower the kernel's shared-memory limit
    below what a larger launch on another context needs."""
    small = I.config_batch("j30_batch", 8)
    big = I.config_batch("j120_batch", 3)
    ids = solver.load(small)
    solver.search_noalloc(ids, iterations=30, delta=20, tabu_len=60, mode=R.EVAL_TIME)
    solver.results(ids)
    with R.Solver(0) as other:
        bid = other.load(big)
        other.search(bid, iterations=30, delta=60, tabu_len=800, mode=R.EVAL_TIME, group_size=8,
                     warps_per_cta=16)
        got = other.results(bid)
    ref = oracle.tabu_search_batch(big, [(30, 60, 800, oracle.TIME, 1)] * len(big), NPROC)
    for g, r in zip(got, ref):
        same_as_oracle(g, r)
    solver.free(ids)
