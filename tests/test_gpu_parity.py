"""GPU parity: the CUDA path against the CPU reference, bit-exact.

Integer results must be identical: every decoded start time and makespan,
the work counters, the whole tabu trajectory (u, v, C per iteration), the
best list, its schedule, the makespan and the number of evaluated
neighbours.  Sizes span several CTAs, group shapes and ragged stripes.
"""
import os

import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R
from test_oracle_pins import medium_instances, random_feasible_list

pytestmark = pytest.mark.gpu

NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module")
def solver():
    from paper_1711_04556_gb300 import build as B
    B.build()
    s = R.Solver(0)
    yield s
    s.close()


def compare_search(oracle, gpu, ref, trace_gpu=None):
    assert gpu["status"] == 0
    assert gpu["best_cmax"] == ref["best_cmax"]
    assert gpu["iterations"] == ref["iterations"]
    assert gpu["evaluated"] == ref["evaluated"]
    assert gpu["work"] == ref["work"]
    assert gpu["best_W"].tolist() == ref["best_W"].tolist()
    assert gpu["best_S"].tolist() == ref["best_S"].tolist()
    assert gpu["cp"] == ref["cp"] and gpu["mode"] == ref["mode"]
    if trace_gpu is not None:
        assert trace_gpu.tolist() == ref["trace"].tolist()


# ----------------------------------------------------------------- decoders
def test_table1_decode(solver, oracle):
    from golden import fixtures
    text, vals = fixtures.read("table1_instance.txt")
    inst = I.Instance.from_text(text)
    ids = solver.load([inst])
    for mode in (R.EVAL_TIME, R.EVAL_CAPACITY):
        cmax, S, work = solver.evaluate_lists(ids[0], np.array([vals["W"]], np.int32), mode)
        ref = oracle.decode(inst, vals["W"], mode)
        assert cmax[0] == 22 and S[0].tolist() == ref[1].tolist() and work[0] == ref[2]
    solver.free(ids)


def wide_instances(count, first=0):
    """Demands up to 200, so capacities exceed 127 (16-bit profile fields); M in
    {1, 2, 3, 5, 8} gives 1, 2 and 4 profile words per time step."""
    ms = (1, 2, 3, 5, 8)
    return [I.generate(s, 12 + s % 25, ms[s % 5], 150 + 30 * (s % 3), 20 + 40 * (s % 3),
                       dmax=4 + s % 7, rmax=200, relabel=bool(s % 2), stream=31)
            for s in range(first, first + count)]


@pytest.mark.parametrize("family", ["medium", "j30", "j120", "mixed", "wide"])
def test_decoders_on_random_lists(solver, oracle, family):
    rng = np.random.default_rng(17)
    insts = {"medium": medium_instances(24, first=900),
             "j30": I.config_batch("j30_batch", 12),
             "j120": I.config_batch("j120_batch", 4),
             "mixed": I.config_batch("mixed_batch", 12),
             "wide": wide_instances(15)}[family]
    ids = solver.load(insts)
    for inst, i in zip(insts, ids):
        lists = np.stack([random_feasible_list(inst, rng) for _ in range(5)])
        for mode in (R.EVAL_TIME, R.EVAL_CAPACITY):
            cmax, S, work = solver.evaluate_lists(i, lists, mode)
            for k in range(len(lists)):
                c, s, w = oracle.decode(inst, lists[k], mode)
                assert cmax[k] == c and S[k].tolist() == s.tolist() and work[k] == w
    solver.free(ids)


# ---------------------------------------------------------------- searches
@pytest.mark.parametrize("G", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("mode", [R.EVAL_TIME, R.EVAL_CAPACITY])
def test_single_instance_search_all_group_sizes(solver, oracle, G, mode):
    inst = I.config_batch("j30_single")[0]
    ref = oracle.tabu_search(inst, 100, 20, 60, mode, 1, trace=True)
    ids = solver.load([inst])
    for warps in ((1, 2, 4) if G <= 2 else (1, 3, 8)):
        solver.search(ids, iterations=100, delta=20, tabu_len=60, mode=mode, group_size=G,
                      warps_per_cta=warps, trace=True)
        res = solver.results(ids)[0]
        compare_search(oracle, res, ref, solver.trace(ids[0], 100))
    solver.free(ids)


def test_j30_batch_full_size(solver, oracle):
    """The 480-instance, 1000-iteration workload in the default launch shape."""
    insts = I.config_batch("j30_batch")
    ids = solver.load(insts)
    solver.search(ids, iterations=1000, delta=20, tabu_len=60, mode=R.EVAL_AUTO)
    got = solver.results(ids)
    ref = oracle.tabu_search_batch(insts, [(1000, 20, 60, 0, 1)] * len(insts), NPROC)
    for g, r in zip(got, ref):
        compare_search(oracle, g, r)
    solver.free(ids)


@pytest.mark.parametrize("mode", [R.EVAL_TIME, R.EVAL_CAPACITY])
def test_j120_sample(solver, oracle, mode):
    insts = I.config_batch("j120_batch", 10)
    ids = solver.load(insts)
    solver.search(ids, iterations=60, delta=60, tabu_len=800, mode=mode, trace=True)
    got = solver.results(ids)
    ref = oracle.tabu_search_batch(insts, [(60, 60, 800, mode, 1)] * len(insts), NPROC, trace=True)
    for k, (g, r) in enumerate(zip(got, ref)):
        compare_search(oracle, g, r, solver.trace(ids[k], 60))
    solver.free(ids)


@pytest.mark.parametrize("mode", [R.EVAL_TIME, R.EVAL_CAPACITY])
def test_wide_fields_search(solver, oracle, mode):
    insts = wide_instances(10, first=40)
    assert max(int(x.cap.max()) for x in insts) > 127
    ids = solver.load(insts)
    solver.search(ids, iterations=40, delta=8, tabu_len=15, mode=mode, trace=True)
    got = solver.results(ids)
    ref = oracle.tabu_search_batch(insts, [(40, 8, 15, mode, 1)] * len(insts), NPROC, trace=True)
    for k, (g, r) in enumerate(zip(got, ref)):
        compare_search(oracle, g, r, solver.trace(ids[k], 40))
    solver.free(ids)


def test_mixed_sample_auto(solver, oracle):
    insts = I.config_batch("mixed_batch", 20)
    ids = solver.load(insts)
    solver.search(ids, iterations=12, delta=0, tabu_len=0, mode=R.EVAL_AUTO)
    got = solver.results(ids)
    params = [(12,) + I.search_params(x.n - 2) + (0, 1) for x in insts]
    ref = oracle.tabu_search_batch(insts, params, NPROC)
    for g, r in zip(got, ref):
        compare_search(oracle, g, r)
    solver.free(ids)


def test_autotuned_shape_keeps_results(solver, oracle, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("RCPSP_TUNE_CACHE", str(cache))
    insts = I.config_batch("j30_batch", 64, first=300)
    ids = solver.load(insts)
    g, w, cs = solver.autotune(ids, iterations=80, delta=20, tabu_len=60, trial_iterations=8)
    lines = cache.read_text().strip().splitlines()
    assert lines and lines[-1].split("\t")[2].split() == [str(g), str(w), str(cs)]
    assert cs in (1, 2, 4, 8)
    with R.Solver(0) as other:                       # a new context reads the table back
        assert other.lib.rcpsp_last_error(other.ctx) is not None
    assert g in (1, 2, 4, 8, 16, 32) and 1 <= w <= 16
    solver.search(ids, iterations=80, delta=20, tabu_len=60)            # shape 0/0: the tuned one
    got = solver.results(ids)
    ref = oracle.tabu_search_batch(insts, [(80, 20, 60, 0, 1)] * len(insts), NPROC)
    for a, b in zip(got, ref):
        compare_search(oracle, a, b)
    solver.free(ids)


@pytest.mark.parametrize("csize", [2, 4, 8])
def test_cluster_split_search(solver, oracle, csize):
    """One search per cluster of CTAs: neighbourhood split, keys exchanged
    through distributed shared memory; results unchanged."""
    single = I.config_batch("j30_single")
    j120 = I.config_batch("j120_batch", 6, first=30)
    mixed = [x for x in I.config_batch("mixed_batch", 24) if x.n <= 122][:6]
    for insts, it, dl, tl, mode in ((single, 100, 20, 60, R.EVAL_TIME), (j120, 30, 60, 800, R.EVAL_AUTO),
                                    (j120, 30, 60, 800, R.EVAL_CAPACITY), (mixed, 10, 0, 0, R.EVAL_AUTO)):
        ids = solver.load(insts)
        solver.search(ids, iterations=it, delta=dl, tabu_len=tl, mode=mode, cluster_size=csize, trace=True)
        got = solver.results(ids)
        params = []
        for x in insts:
            d_, t_ = (dl, tl) if dl else I.search_params(x.n - 2)
            params.append((it, d_, t_, mode, 1))
        ref = oracle.tabu_search_batch(insts, params, NPROC, trace=True)
        for k, (g, r) in enumerate(zip(got, ref)):
            compare_search(oracle, g, r, solver.trace(ids[k], it))
        solver.free(ids)


def test_multistart_keeps_the_best_start(solver, oracle):
    from paper_1711_04556_gb300.multistart import multistart
    inst = I.config_batch("j30_batch", 1, first=123)[0]
    out = multistart(solver, inst, starts=8, seed=5, iterations=60, delta=20, tabu_len=60)
    refs = [oracle.tabu_search(inst, 60, 20, 60, 0, 1, level_key=k) for k in out["keys"]]
    assert out["makespans"] == [r["best_cmax"] for r in refs]
    best = min(range(8), key=lambda k: (refs[k]["best_cmax"], k))
    assert out["start"] == best and out["best_W"].tolist() == refs[best]["best_W"].tolist()


def test_bounded_wait_reports_timeout(solver, monkeypatch):
    """A host wait with a tiny limit returns RCPSP_E_TIMEOUT instead of
    blocking; the context stays usable and a later wait succeeds."""
    import time
    insts = I.config_batch("j30_batch", 240, first=600)
    ids = solver.load(insts)
    monkeypatch.setenv("RCPSP_WAIT_SECONDS", "0")
    solver.search(ids, iterations=1000, delta=20, tabu_len=60)
    with pytest.raises(R.RcpspError) as e:
        solver.results(ids)
    assert e.value.code == -7
    monkeypatch.setenv("RCPSP_WAIT_SECONDS", "300")
    time.sleep(0.2)
    assert all(r["status"] == 0 for r in solver.results(ids))
    solver.free(ids)


# -------------------------------------------------------------- edge cases
def test_edge_cases(solver, oracle):
    base = medium_instances(1, first=1000)[0]
    big = np.array([base.req[k::base.m].sum() + 1 for k in range(base.m)], np.int32)
    free = I.Instance(base.n, base.m, base.dur, big, base.req, base.succ_off, base.succ)
    n = 5
    succ_sets = [[1]] + [[i + 1] for i in range(1, n + 1)] + [[]]
    off = np.r_[0, np.cumsum([len(s) for s in succ_sets])].astype(np.int32)
    chain = I.Instance(n + 2, 1, np.r_[0, np.full(n, 2), 0].astype(np.int32), np.array([1], np.int32),
                       np.r_[0, np.ones(n), 0].astype(np.int32), off,
                       np.array([x for s in succ_sets for x in s], np.int32))
    one = I.generate(2, 1, 2, 150, 50, stream=11)            # N = 3: no moves at all
    relab = I.generate(5, 14, 3, 210, 20, relabel=True, stream=11)
    cases = [(free, (40, 6, 5, 1, 1)), (chain, (7, 4, 3, 1, 0)), (one, (5, 3, 2, 2, 0)),
             (relab, (25, 1, 1, 1, 0)), (relab, (25, 50, 1, 2, 0)), (base, (0, 5, 5, 1, 1)),
             (base, (30, 3, 200, 2, 0))]
    for inst, (it, dl, tl, mode, stop) in cases:
        ids = solver.load([inst])
        solver.search(ids, iterations=it, delta=dl, tabu_len=tl, mode=mode, stop_at_cp=bool(stop), trace=True)
        ref = oracle.tabu_search(inst, it, dl, tl, mode, stop, trace=True)
        compare_search(oracle, solver.results(ids)[0], ref, solver.trace(ids[0], max(it, 1)))
        solver.free(ids)


def test_level_keys_and_repeat_with_graph(solver, oracle):
    import torch
    insts = I.config_batch("j30_batch", 40, first=100)
    keys = [I.level_keys(x, k) for k, x in enumerate(insts)]
    ids = solver.load(insts, keys)
    st = torch.cuda.Stream()
    outs = []
    for _ in range(3):
        solver.search(ids, iterations=50, delta=20, tabu_len=60, use_graph=True, stream=st)
        outs.append(solver.results(ids))
    ref = oracle.tabu_search_batch(insts, [(50, 20, 60, 0, 1)] * len(insts), NPROC, level_keys=keys)
    for o in outs:
        for g, r in zip(o, ref):
            compare_search(oracle, g, r)
    solver.free(ids)


def test_kernel_launch_count(solver):
    """One kernel per launch class of a search; graph replays count too."""
    insts = I.config_batch("j30_batch", 8) + [x for x in I.config_batch("mixed_batch", 40) if x.n == 302][:1]
    ids = solver.load(insts)
    k0 = solver.kernel_launches()
    solver.search(ids[:8], iterations=5)
    assert solver.kernel_launches() - k0 == 1
    import torch
    st = torch.cuda.Stream()
    solver.search(ids, iterations=5, use_graph=True, stream=st)
    solver.search(ids, iterations=5, use_graph=True, stream=st)
    assert solver.kernel_launches() - k0 == 5          # two classes, twice
    solver.results(ids)
    solver.free(ids)


@pytest.mark.parametrize("mode", [R.EVAL_TIME, R.EVAL_CAPACITY])
def test_prefix_reuse_and_full_decodes_agree(solver, oracle, mode):
    """Prefix reuse is used when an iteration needs several decode rounds:
    few groups (G = 8 x 2 warps: 8 groups for ~850 feasible moves) run the
    kernel variant that starts neighbour decodes from kept states, many
    groups (48 per CTA on clusters of 8 CTAs: 384) the one that decodes
    from the start.  Both must be the oracle's search."""
    insts = I.config_batch("j120_batch", 6, first=90)
    ids = solver.load(insts)
    ref = oracle.tabu_search_batch(insts, [(12, 60, 800, mode, 1)] * len(insts), NPROC, trace=True)
    for g, w, c in ((8, 2, 1), (8, 12, 8)):
        solver.search(ids, iterations=12, delta=60, tabu_len=800, mode=mode, group_size=g, warps_per_cta=w,
                      cluster_size=c, trace=True)
        got = solver.results(ids)
        for k, (a, b) in enumerate(zip(got, ref)):
            compare_search(oracle, a, b, solver.trace(ids[k], 12))
    solver.free(ids)


def test_largest_sizes_and_zero_durations(solver, oracle):
    """N = 302 with 8 resources and durations up to 50 (the longest horizon),
    the largest tabu list, non-dummy activities of zero duration, and an
    empty call."""
    big = I.generate(17, 300, 8, 180, 50, dmin=1, dmax=50, stream=41)
    zero_dur = I.config_batch("j30_batch", 1, first=77)[0]
    d = zero_dur.dur.copy()
    d[1:-1:4] = 0
    zero = I.Instance(zero_dur.n, zero_dur.m, d, zero_dur.cap, zero_dur.req, zero_dur.succ_off, zero_dur.succ)
    for inst, it, dl, tl in ((big, 2, 60, 8192),             # 8192 = RCPSP_MAX_TABU
                             (zero, 40, 20, 60)):
        for mode in (R.EVAL_TIME, R.EVAL_CAPACITY):
            ids = solver.load([inst])
            solver.search(ids, iterations=it, delta=dl, tabu_len=tl, mode=mode, trace=True)
            ref = oracle.tabu_search(inst, it, dl, tl, mode, 1, trace=True)
            compare_search(oracle, solver.results(ids)[0], ref, solver.trace(ids[0], it))
            solver.free(ids)
    solver.search([], iterations=5)
    assert solver.results([]) == []


def test_launch_shape_limits(solver, oracle):
    """CTAs of up to 12 warps run the 384-thread build of the search kernel,
    13 to 16 warps the 512-thread build: both give the oracle's searches.
    17 warps is refused as an invalid parameter."""
    insts = I.config_batch("j30_batch", 6, first=31)
    ids = solver.load(insts)
    ref = oracle.tabu_search_batch(insts, [(30, 20, 60, 0, 1)] * len(insts), NPROC)
    for w in (12, 13, 16):
        solver.search(ids, iterations=30, delta=20, tabu_len=60, group_size=2, warps_per_cta=w)
        for g, r in zip(solver.results(ids), ref):
            assert g["best_cmax"] == r["best_cmax"] and g["evaluated"] == r["evaluated"]
            assert g["best_W"].tolist() == r["best_W"].tolist()
    for bad in (17, -1):
        with pytest.raises(R.RcpspError) as e:
            solver.search(ids, iterations=5, delta=20, tabu_len=60, warps_per_cta=bad)
        assert e.value.code == -1
    with pytest.raises(R.RcpspError) as e:
        solver.coop_search(ids, iterations=5, blocks=2, working_set=2, phi_steps=0, warps_per_cta=17)
    assert e.value.code == -1
    solver.free(ids)
