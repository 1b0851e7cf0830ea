"""The layer-skipping instance family (tests/skip_arc_instances.py) against
the problem statement (Sec. 2), and the CPU reference on it."""
import numpy as np

from paper_1711_04556_gb300 import rcpsp as R
from skip_arc_instances import reachable, skip_arc_batch, with_skip_arcs


def test_skip_arc_instances_follow_the_problem_statement(oracle):
    insts = skip_arc_batch(12) + [with_skip_arcs(s, 120, 4, 180, 20, extra=40, relabel=True) for s in range(2)]
    for x in insts:
        N = x.n
        succ = [set(int(j) for j in x.successors(i)) for i in range(N)]
        preds = [set() for _ in range(N)]
        for a in range(N):
            for b in succ[a]:
                preds[b].add(a)
        assert x.dur[0] == 0 and x.dur[N - 1] == 0
        assert [i for i in range(N) if not preds[i]] == [0]
        assert [i for i in range(N) if not succ[i]] == [N - 1]
        # acyclic, and every arc necessary (no longer path implies it)
        for a in range(N):
            assert not reachable(succ, a, a)
            for b in succ[a]:
                assert not reachable(succ, a, b, skip_arc=(a, b)), (a, b)
        # some arcs join activities whose longest-path levels differ by 2 or more
        lev = [0] * N
        for a in oracle.initial_order(x):
            for b in succ[a]:
                lev[b] = max(lev[b], lev[a] + 1)
        skips = sum(1 for a in range(1, N - 1) for b in succ[a] if b != N - 1 and lev[b] - lev[a] >= 2)
        assert skips >= 1
        # the library's host preparation accepts it and agrees with the oracle
        p = R.prepare(x)
        assert p["cp"] == oracle.critical_path(x) and p["initial"].tolist() == oracle.initial_order(x).tolist()
    relabelled = [x for x in insts if x.meta["relabel"]]
    assert any(any(b < a for a in range(1, x.n - 1) for b in x.successors(a) if b != x.n - 1) for x in relabelled)


def test_oracle_search_on_skip_arcs_is_feasible(oracle):
    for x in skip_arc_batch(6, first=20):
        for mode in (oracle.TIME, oracle.CAPACITY):
            r = oracle.tabu_search(x, 60, 20, 60, mode, 1)
            code, cmax = oracle.check_schedule(x, r["best_S"])     # 0: feasible (Eqs. 2-4)
            assert code == 0 and cmax == r["best_cmax"] >= r["cp"]
            W = r["best_W"]
            pos = np.argsort(W)
            assert all(pos[a] < pos[b] for a in range(x.n) for b in x.successors(a))
