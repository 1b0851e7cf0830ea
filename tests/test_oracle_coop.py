"""Pins of the co-operative search of the CPU reference (Sec. 6.1, Eq. 8).

The co-operation has no printed trajectory either, so its pins are: the
reduction to the single search of Sec. 6 when nothing is exchanged, the
symmetry of identical blocks, closed forms and the mathematical exponential
for Eq. 8, a brute-force restatement of the random feasible swaps, and the
rules the paper states (the working set only improves, reads go round the
set, at least five reads per block, every exchange has its cause).  CPU only.
"""
import math

import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I

from test_oracle_pins import list_is_feasible, medium_instances

BIG = 10**9


def coop(oracle, inst, **kw):
    base = dict(iterations=60, delta=8, tabu_len=15, mode=0, stop_at_cp=1, blocks=4, working_set=8,
                phi_max=3, phi_steps=20, assign_fixed=0)
    base.update(kw)
    if "words" not in base and base["phi_steps"] > 0:
        base["slot_keys"], base["words"] = I.coop_inputs(inst, 3, base["working_set"], base["blocks"], 64)
    return oracle.coop_search(inst, **base)


# ------------------------------------------------------------------ Eq. 8
def test_exp_neg_is_the_exponential(oracle):
    for x in np.concatenate([np.linspace(0, 1, 101), np.linspace(1, 120, 239), [300.0, 699.0]]):
        assert oracle.exp_neg(x) == pytest.approx(math.exp(-x), rel=1e-12, abs=0)
    assert oracle.exp_neg(0.0) == 1.0
    assert oracle.exp_neg(701.0) == 0.0


@pytest.mark.parametrize("i_block", [1, 5, 37, 100, 1000, 5000])
def test_eq8_closed_forms(oracle, i_block):
    # the best solution, never searched: quality = intactness = 1
    assert oracle.assigned_iterations(50, 50, 0, i_block) == i_block // 5
    assert oracle.assigned_iterations(0, 0, 0, i_block) == i_block // 5
    # no iterations for anything when I_block is 0
    assert oracle.assigned_iterations(60, 50, 10, 0) == 0


def test_eq8_against_the_formula(oracle):
    rng = np.random.default_rng(8)
    checked = 0
    for _ in range(3000):
        cs = int(rng.integers(1, 400))
        ck = cs + int(rng.integers(0, 30))
        ib = int(rng.integers(1, 6000))
        ic = int(rng.integers(0, 4 * ib))
        v = ib / 5 * (0.8 * math.exp(-100 * (ck / cs - 1)) + 0.2 * math.exp(-4 * ic / ib))
        if abs(v - round(v)) < 1e-9 * max(1.0, v):
            continue                                     # floor decided by rounding
        assert oracle.assigned_iterations(ck, cs, ic, ib) == math.floor(v)
        checked += 1
    assert checked > 2900


def test_eq8_prefers_good_and_fresh_solutions(oracle):
    a = [oracle.assigned_iterations(100 + k, 100, 0, 1000) for k in range(30)]
    assert all(x >= y for x, y in zip(a, a[1:])) and a[0] == 200 and a[-1] == 40
    b = [oracle.assigned_iterations(100, 100, ic, 1000) for ic in range(0, 5000, 250)]
    assert all(x >= y for x, y in zip(b, b[1:])) and b[-1] == 160


# ---------------------------------------------------------- diversification
def feasible_moves(oracle, inst, W, delta):
    return [(u, v) for u in range(1, inst.n - 1) for v in range(u + 1, min(inst.n - 2, u + delta) + 1)
            if oracle.move_feasible(inst, W, u, v)]


def test_diversify_takes_the_drawn_feasible_swaps(oracle):
    rng = np.random.default_rng(4)
    for inst in medium_instances(6):
        W0 = oracle.initial_order(inst)
        words = rng.integers(0, 2**32, 7, dtype=np.uint64).astype(np.uint32)
        for steps, cursor in ((0, 0), (1, 3), (5, 6), (20, 2)):
            W, done, cur = oracle.diversify(inst, W0, 6, steps, words, cursor)
            ref = np.array(W0)
            c = cursor
            for _ in range(steps):
                mv = feasible_moves(oracle, inst, ref, 6)
                if not mv:
                    break
                w = int(words[c % len(words)])
                c += 1
                u, v = mv[(w * len(mv)) >> 32]
                ref[u], ref[v] = ref[v], ref[u]
                assert list_is_feasible(inst, ref)
            assert W.tolist() == ref.tolist() and cur == c and done == c - cursor


def test_diversify_without_feasible_swaps(oracle):
    # a chain: every swap breaks an arc, so nothing is drawn
    n = 7
    succ_off = np.array([0, 1, 2, 3, 4, 5, 6, 6], np.int32)
    succ = np.array([1, 2, 3, 4, 5, 6], np.int32)
    chain = I.Instance(n, 1, np.array([0, 1, 2, 3, 1, 2, 0], np.int32), np.array([3], np.int32),
                       np.array([0, 1, 1, 1, 1, 1, 0], np.int32), succ_off, succ)
    W, done, cur = oracle.diversify(chain, np.arange(n), 3, 20, np.arange(5, dtype=np.uint32), 2)
    assert W.tolist() == list(range(n)) and done == 0 and cur == 2


# ------------------------------------------------------ whole co-operation
@pytest.mark.parametrize("mode", [1, 2])
def test_single_block_without_exchanges_is_the_plain_search(oracle, mode):
    """B = |F| = 1, reads never diversified and never timed out: every
    exchange writes the block's own list back and reads it again, so the
    search is the single search of Sec. 6, step for step."""
    for inst in medium_instances(6, first=20):
        for it in (0, 1, 45):
            ref = oracle.tabu_search(inst, it, 8, 15, mode, 1)
            got = coop(oracle, inst, iterations=it, mode=mode, blocks=1, working_set=1, phi_max=BIG,
                       phi_steps=0, assign_fixed=it + 1)
            for k in ("best_cmax", "iterations", "evaluated", "work", "status", "cp", "mode"):
                assert got[k] == ref[k], k
            assert got["best_W"].tolist() == ref["best_W"].tolist()
            assert got["best_S"].tolist() == ref["best_S"].tolist()


def test_identical_blocks_run_identical_searches(oracle):
    """B blocks reading B identical slots with identical random words each
    repeat the one-block search (its exchanges included) exactly."""
    for inst in medium_instances(4, first=40):
        _, words = I.coop_inputs(inst, 9, 1, 1, 32)
        one = coop(oracle, inst, iterations=80, blocks=1, working_set=1, phi_max=1, phi_steps=4,
                   slot_keys=None, words=words, stop_at_cp=0, fbi_every=0)
        for b in (2, 3):
            many = coop(oracle, inst, iterations=80, blocks=b, working_set=b, phi_max=1, phi_steps=4,
                        slot_keys=None, words=np.repeat(words, b, axis=0), stop_at_cp=0, fbi_every=0)
            assert many["best_cmax"] == one["best_cmax"]
            assert many["best_W"].tolist() == one["best_W"].tolist()
            assert many["evaluated"] == b * one["evaluated"] and many["work"] == b * one["work"]
            assert many["iterations"] == b * one["iterations"]


@pytest.mark.parametrize("blocks,fsize,phi_max", [(4, 8, 1), (3, 2, 0), (5, 16, 3)])
def test_exchange_rules(oracle, blocks, fsize, phi_max):
    for inst in medium_instances(3, first=60):
        ib = 100
        r = coop(oracle, inst, iterations=ib, blocks=blocks, working_set=fsize, phi_max=phi_max,
                 stop_at_cp=0, log_cap=100000)
        assert r["status"] == 0 and r["iterations"] == blocks * ib
        log = r["log"]
        assert len(log) == r["log_events"]
        slot_c = {}
        reads = [e for e in log if e["kind"] == 2]
        # reads go round the working set
        assert [e["slot"] for e in reads] == [k % fsize for k in range(len(reads))]
        for e in reads:
            assert 0 <= e["assigned"] <= ib // 5
            assert (e["diversified"] > 0) == (e["phi"] > phi_max)
        # at least five reads per block (Sec. 6.1)
        for b in range(blocks):
            mine = [e for e in reads if e["block"] == b]
            assert len(mine) >= 5
            # no read lasts more than its assigned iterations + 1
            its = [e["iteration"] for e in mine]
            for e, nxt in zip(mine, its[1:]):
                assert nxt - max(e["iteration"], 0) <= e["assigned"] + 1
        # the working set only improves, and never above what was read
        for e in log:
            if e["kind"] == 1:
                assert e["cmax"] < slot_c.get(e["slot"], 1 << 30)
                slot_c[e["slot"]] = e["cmax"]
                assert e["phi"] == 0
        writes = [e["cmax"] for e in log if e["kind"] == 1]
        assert r["best_cmax"] <= min(writes + [1 << 30]) and r["best_cmax"] >= r["cp"]
        rc, cm = oracle.check_schedule(inst, r["best_S"])
        assert rc == 0 and cm == r["best_cmax"]


def test_cooperation_stops_at_the_critical_path(oracle):
    inst = I.generate(11, 12, 2, 150, 100, stream=31)       # RS = 1: every list meets the CP
    r = coop(oracle, inst, iterations=50, blocks=4, working_set=4)
    assert r["best_cmax"] == r["cp"] and r["iterations"] == 0 and r["evaluated"] == 0


def test_cooperation_is_no_worse_than_its_first_slot(oracle):
    """The result is never worse than the plain search from slot 0's list
    would be at the start, and it is a feasible schedule."""
    for inst in I.config_batch("j30_batch", 6, first=200):
        keys, words = I.coop_inputs(inst, 1, 8, 4, 64)
        r = oracle.coop_search(inst, 50, 20, 60, 0, 1, 4, 8, 3, 20, 0, keys, words)
        c0 = oracle.decode(inst, oracle.initial_order(inst), r["mode"])[0]
        assert r["status"] == 0 and r["cp"] <= r["best_cmax"] <= c0
        rc, cm = oracle.check_schedule(inst, r["best_S"])
        assert rc == 0 and cm == r["best_cmax"]


# ------------------------------------------------------------------- FBI
def test_fbi_backward_schedule_is_a_schedule(oracle):
    """The backward pass, mirrored, is a feasible schedule of the original
    instance (independent checker) no longer than the forward one (TIME:
    the serial SGS right-justifies); the forward pass is no longer than it."""
    rng = np.random.default_rng(17)
    from test_oracle_pins import random_feasible_list
    insts = medium_instances(8, first=80) + I.config_batch("j30_batch", 6, first=30)
    for inst in insts:
        for _ in range(4):
            W = random_feasible_list(inst, rng)
            for mode in (1, 2):
                c = oracle.decode(inst, W, mode)[0]
                Wn, c2, T, Sb = oracle.fbi_pass(inst, W, mode)
                rc, cm = oracle.check_schedule(inst, Sb)
                assert rc == 0 and cm == T
                assert list_is_feasible(inst, Wn)
                assert sorted(Wn.tolist()) == list(range(inst.n))
                assert [Sb[a] for a in Wn] == sorted(Sb.tolist())      # forward list by backward start
                if mode == 1:
                    assert T <= c and c2 <= T


def test_fbi_never_worse_and_converged(oracle):
    rng = np.random.default_rng(5)
    from test_oracle_pins import random_feasible_list
    improved = 0
    for inst in medium_instances(6, first=90) + I.config_batch("j30_batch", 8, first=60):
        for mode in (1, 2):
            W = random_feasible_list(inst, rng)
            c0 = oracle.decode(inst, W, mode)[0]
            Wf, c, passes = oracle.fbi(inst, W, mode)
            assert c <= c0 and (passes > 0) == (c < c0)
            assert oracle.decode(inst, Wf, mode)[0] == c and list_is_feasible(inst, Wf)
            again, c1, p1 = oracle.fbi(inst, Wf, mode)                  # a fixed point
            assert p1 == 0 and c1 == c and again.tolist() == Wf.tolist()
            improved += c < c0
    assert improved > 0


def test_fbi_not_below_the_optimum(oracle):
    from test_oracle_pins import small_instances
    for inst in small_instances(12, n=6):
        opt = oracle.brute_force_starts(inst)
        W = oracle.initial_order(inst)
        for mode in (1, 2):
            assert oracle.fbi(inst, W, mode)[1] >= opt
