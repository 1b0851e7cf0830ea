"""The search without device allocation (rcpsp_tabu_search_noalloc).

Some callers cannot allocate device memory when they search -- a serving
process whose device memory belongs to another allocator with a fixed
budget, or a host thread that may not wait on the device synchronisation
that cudaMalloc / cudaFree can imply.  For them the library offers a
variant of the search launch whose plan and work-queue counter live in a
fixed array inside the library.  Through the C interface it must give the
same results as rcpsp_tabu_search, on two calls in a row (the second call
finds the array holding the first call's plan and counter).

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R

pytestmark = pytest.mark.gpu

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


def test_noalloc_matches_allocating_search_twice(solver):
    import torch
    insts = I.config_batch("j30_batch", 64, first=200) + I.config_batch("j120_batch", 4)
    ids = solver.load(insts)
    st = torch.cuda.Stream()
    kw = dict(iterations=120, delta=0, tabu_len=0, mode=R.EVAL_AUTO)
    solver.search(ids, stream=st, **kw)
    ref = solver.results(ids)
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


def test_noalloc_limits(solver):
    ids = solver.load(I.config_batch("j30_single"))
    params = R.Params(10, 0, 0, 0, 1, 0, 0, 0, 0)
    too_many = np.zeros(9361, np.int32)               # one more than the array holds
    rc = solver.lib.rcpsp_tabu_search_noalloc(solver.ctx, R._ptr(too_many), too_many.size, R.C.byref(params), None)
    assert rc == -5
    traced = R.Params(10, 0, 0, 0, 1, 0, 0, 1, 0)    # record_trace = 1
    one = np.asarray(ids, np.int32)
    rc = solver.lib.rcpsp_tabu_search_noalloc(solver.ctx, R._ptr(one), 1, R.C.byref(traced), None)
    assert rc == -1
    solver.free(ids)
