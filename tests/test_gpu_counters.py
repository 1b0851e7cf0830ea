"""Work counters of the decodes (rcpsp_stats.placements .. kept_words).

The throughput accounting of the benchmark divides the work the kernel
actually performed by its time, so these counters must be exact.  Without
prefix reuse every neighbour is decoded from the first position: the
counters are closed forms of the number of evaluated neighbours.  With
prefix reuse a neighbour (u, v) restores the current list's decoder state
before position floor(u/K)*K (at most (N-1)//K states, K = max(8,
ceil(N/32))) and places only the positions from there on, and every
iteration decodes the current list once to produce those states; the test
replays the traced trajectory on the CPU, enumerates every iteration's
feasible moves with the CPU reference (Eqs. 5-6) and recomputes the
placements, Alg. 6 update steps and successor pushes from those definitions.
"""
import os

import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R

pytestmark = pytest.mark.gpu

NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def solver():
    from paper_1711_04556_gb300 import build as B
    B.build()
    s = R.Solver(0)
    yield s
    s.close()


def used(inst):
    return np.count_nonzero(inst.req.reshape(inst.n, inst.m), axis=1)


@pytest.mark.parametrize("mode", [R.EVAL_TIME, R.EVAL_CAPACITY])
def test_counters_without_prefix_reuse(solver, mode):
    insts = I.config_batch("j30_batch", 24)
    ids = solver.load(insts)
    # one decode round per iteration: the launch keeps prefix reuse off
    solver.search(ids, iterations=60, delta=20, tabu_len=60, mode=mode, group_size=4, warps_per_cta=12,
                  cluster_size=1)
    for x, r in zip(insts, solver.results(ids)):
        ev = r["evaluated"]
        per_upd = int(x.dur.sum()) if mode == R.EVAL_TIME else int(used(x).sum())
        assert r["placements"] == ev * x.n
        assert r["steps_done"] == r["work"]
        assert r["update_units"] == ev * per_upd
        assert r["succ_pushes"] == ev * int(x.succ_off[-1])
        assert r["kept_words"] == 0
    solver.free(ids)


@pytest.mark.parametrize("mode", [R.EVAL_TIME, R.EVAL_CAPACITY])
def test_counters_with_prefix_reuse(solver, oracle, mode):
    insts = I.config_batch("j120_batch", 3)
    iters = 25
    ids = solver.load(insts)
    # four decoding groups for ~100+ feasible moves: several decode rounds,
    # so the launch keeps decoder states of the current list
    solver.search(ids, iterations=iters, delta=60, tabu_len=800, mode=mode, group_size=8, warps_per_cta=1,
                  cluster_size=1, trace=True)
    res = solver.results(ids)
    for k, (x, r) in enumerate(zip(insts, res)):
        n = x.n
        K = max(8, (n + 31) // 32)
        count = (n - 1) // K
        per = x.dur.astype(np.int64) if mode == R.EVAL_TIME else used(x).astype(np.int64)
        nsucc = np.diff(x.succ_off).astype(np.int64)
        W = np.asarray(R.prepare(x)["initial"], np.int32).copy()
        placed = upd = succ = ev = 0
        tr = solver.trace(ids[k], r["iterations"])
        for u_star, v_star, _ in tr:
            # the producer decodes the current list in full
            placed += n
            upd += int(per.sum())
            succ += int(nsucc.sum())
            pre_upd = np.concatenate([[0], np.cumsum(per[W])])
            pre_succ = np.concatenate([[0], np.cumsum(nsucc[W])])
            for u in range(1, n - 2):
                for v in range(u + 1, min(u + 60, n - 2) + 1):
                    if not oracle.move_feasible(x, W, u, v):
                        continue
                    ev += 1
                    p0 = min(u // K, count) * K
                    placed += n - p0
                    upd += int(pre_upd[-1] - pre_upd[p0])
                    succ += int(pre_succ[-1] - pre_succ[p0])
            if u_star or v_star:
                W[u_star], W[v_star] = W[v_star], W[u_star]
        assert ev == r["evaluated"]
        assert r["placements"] == placed
        assert r["update_units"] == upd
        assert r["succ_pushes"] == succ
        assert r["placements"] < (r["evaluated"] + r["iterations"]) * n
        assert 0 < r["kept_words"]
        assert 0 < r["steps_done"]
    solver.free(ids)
