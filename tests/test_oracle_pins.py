"""Pins of the CPU reference (oracle) to facts outside itself.

Each test ties an oracle routine to something the paper or mathematics
fixes: the worked example of Table 1, the update example of Fig. 4,
independent definitions (list feasibility, path enumeration, the sequential
upper envelope behind the capacity-indexed state, exact earliest fit), brute
force over all lists and over left-justified start vectors, and special
cases with closed forms.  CPU only.
"""
import numpy as np
import pytest

from golden import fixtures
from paper_1711_04556_gb300.instances import Instance, generate, table1_instance


# ----------------------------------------------------------------- helpers
def list_is_feasible(inst, W):
    """A list is precedence-feasible iff every arc points forward in it."""
    pos = np.empty(inst.n, np.int64)
    pos[np.asarray(W)] = np.arange(inst.n)
    return all(pos[i] < pos[j] for i, j in inst.arcs())


def random_feasible_list(inst, rng):
    """Random topological order with 0 first and N-1 last."""
    preds = {j: set() for j in range(inst.n)}
    for i, j in inst.arcs():
        preds[j].add(i)
    done, W = {0}, [0]
    while len(W) < inst.n - 1:
        ready = [i for i in range(1, inst.n - 1) if i not in done and preds[i] <= done]
        i = ready[rng.integers(0, len(ready))]
        W.append(i)
        done.add(i)
    W.append(inst.n - 1)
    return np.array(W, np.int32)


def all_paths(inst, src, dst):
    out, stack = [], [(src, [src])]
    while stack:
        i, path = stack.pop()
        if i == dst:
            out.append(path)
            continue
        for j in inst.successors(i):
            stack.append((int(j), path + [int(j)]))
    return out


def es_by_paths(inst):
    """Earliest starts with unlimited capacity: heaviest path 0 -> j."""
    return [max(sum(int(inst.dur[x]) for x in p[:-1]) for p in all_paths(inst, 0, j))
            for j in range(inst.n)]


def small_instances(count, n=5, m=2, dmax=4, rmax=4, relabel=True, first=0):
    return [generate(s, n, m, 150 + 30 * (s % 3), 20 + 30 * (s % 3), dmax=dmax, rmax=rmax,
                     relabel=relabel, stream=99) for s in range(first, first + count)]


def medium_instances(count, first=0):
    return [generate(s, 8 + s % 17, 1 + s % 4, 150 + 30 * (s % 3), 10 + 30 * (s % 4),
                     dmax=3 + s % 8, rmax=2 + s % 9, relabel=bool(s % 2), stream=98)
            for s in range(first, first + count)]


def table1():
    text, vals = fixtures.read("table1_instance.txt")
    return Instance.from_text(text), vals


# ------------------------------------------------------------ Table 1 pins
def test_table1_fixture_matches_generator_copy():
    inst, _ = table1()
    assert inst.digest() == table1_instance().digest()


def test_table1_critical_path(oracle):
    inst, vals = table1()
    assert oracle.critical_path(inst) == vals["cp"][0] == 16


@pytest.mark.parametrize("mode", [1, 2])
def test_table1_order_makespan(oracle, mode):
    inst, vals = table1()
    W = np.array(vals["W"], np.int32)
    assert list_is_feasible(inst, W)
    cmax, S, _ = oracle.decode(inst, W, mode)
    assert cmax == vals["cmax"][0] == 22
    rc, c2 = oracle.check_schedule(inst, S)
    assert rc == 0 and c2 == 22 and S[inst.n - 1] == 22
    # the start times themselves (the example's resource chart is a figure): the
    # serial SGS restated by earliest fit gives the same schedule
    assert S.tolist() == sgs_earliest_fit(inst, W)[1].tolist()


def test_table1_optimum_by_both_brute_forces(oracle):
    inst, vals = table1()
    best_lists, n_lists = oracle.brute_force_lists(inst, oracle.TIME)
    assert best_lists == oracle.brute_force_starts(inst)
    assert best_lists <= vals["cmax"][0]
    assert best_lists >= vals["cp"][0]
    assert n_lists == count_linear_extensions(inst)


def count_linear_extensions(inst):
    """Number of precedence-feasible lists, by dynamic programming over the
    sets of already listed non-dummy activities."""
    mid = list(range(1, inst.n - 1))
    pred_mask = {i: 0 for i in mid}
    for a, b in inst.arcs():
        if a in pred_mask and b in pred_mask:
            pred_mask[b] |= 1 << mid.index(a)
    full = (1 << len(mid)) - 1
    ways = {full: 1}
    for mask in range(full - 1, -1, -1):
        ways[mask] = sum(ways[mask | (1 << x)] for x, i in enumerate(mid)
                         if not (mask >> x) & 1 and (pred_mask[i] & ~mask) == 0)
    return ways[0]


# ------------------------------------------------------------- Fig. 4 pins
def test_fig4_update(oracle):
    _, v = fixtures.read("fig4_update.txt")
    out, steps = oracle.capacity_update(v["c_before"], v["R"][0], v["r"][0], v["d"][0], v["s"][0])
    assert out.tolist() == v["c_after"]
    # the contributions between the old and the new state add up to r*d
    before = np.array(v["c_before"])
    contrib = [max(0, a - max(b, v["s"][0])) for a, b in zip(out, before) if a != b]
    assert sum(contrib) == v["r"][0] * v["d"][0]
    assert steps == 5


def envelope_update(c, R, r, d, s):
    """Sequential upper envelope: usage u(t) = #{j : c[j] > t}; add r on
    [s, s+d); take the non-increasing envelope; c'[j] = min{t : env(t) <= j}."""
    T = int(max(max(c) if len(c) else 0, s + d)) + 2
    u = np.array([sum(1 for x in c if x > t) for t in range(T)])
    w = u + np.array([r if s <= t < s + d else 0 for t in range(T)])
    env = np.maximum.accumulate(w[::-1])[::-1]
    return np.array([min(t for t in range(T) if env[t] <= j) for j in range(R)])


def test_alg4_equals_upper_envelope(oracle):
    rng = np.random.default_rng(7)
    for _ in range(3000):
        R = int(rng.integers(1, 10))
        c = np.sort(rng.integers(0, 15, R))[::-1]
        r = int(rng.integers(0, R + 1))
        d = int(rng.integers(0, 6))
        s = int((c[R - r] if r else 0) + rng.integers(0, 5))
        out, steps = oracle.capacity_update(c, R, r, d, s)
        assert out.tolist() == envelope_update(list(c), R, r, d, s).tolist()
        assert all(out[j] >= out[j + 1] for j in range(R - 1))
        if r and d:
            contrib = [a - max(b, s) for a, b in zip(out, c) if a != b]
            assert sum(contrib) == r * d
            # the loop runs up to the last entry the update changes
            assert steps == max(j for j in range(R) if out[j] != c[j]) + 1
        else:
            assert out.tolist() == list(c) and steps == 0


# ---------------------------------------------------- decoders: semantics
def decode_by_envelope(inst, W):
    """Capacity-indexed decoding restated on explicit non-increasing usage
    functions: r units of k are free from t on iff env_k(t) + r <= R_k."""
    H = int(inst.dur.sum()) + 2
    env = np.zeros((inst.m, H), np.int64)
    S = np.zeros(inst.n, np.int64)
    preds = {j: [] for j in range(inst.n)}
    for i, j in inst.arcs():
        preds[j].append(i)
    for i in W:
        es = max([S[p] + inst.dur[p] for p in preds[i]], default=0)
        r = inst.req[i * inst.m:(i + 1) * inst.m]
        t = 0
        while any(r[k] > 0 and env[k, t] + r[k] > inst.cap[k] for k in range(inst.m)):
            t += 1
        s = max(es, t)
        S[i] = s
        for k in range(inst.m):
            if r[k] and inst.dur[i]:
                env[k, s:s + inst.dur[i]] += r[k]
                env[k] = np.maximum.accumulate(env[k][::-1])[::-1]
    return int(max(S + inst.dur)), S


def capacity_work_by_envelope(inst, W):
    """Alg. 4 loop steps of a capacity-indexed decode, from explicit usage
    envelopes: per activity and used resource, the capacity-indexed state is
    c[j] = min{t : env(t) <= j}, and the update runs up to the last entry
    it changes."""
    H = int(inst.dur.sum()) + 2
    env = np.zeros((inst.m, H), np.int64)
    S = np.zeros(inst.n, np.int64)
    preds = {j: [] for j in range(inst.n)}
    for i, j in inst.arcs():
        preds[j].append(i)

    def state(e, R):
        return [min(t for t in range(H) if e[t] <= j) for j in range(R)]
    work = 0
    for i in W:
        es = max([S[p] + inst.dur[p] for p in preds[i]], default=0)
        r = inst.req[i * inst.m:(i + 1) * inst.m]
        t = 0
        while any(r[k] > 0 and env[k, t] + r[k] > inst.cap[k] for k in range(inst.m)):
            t += 1
        s = max(es, t)
        S[i] = s
        for k in range(inst.m):
            if r[k] and inst.dur[i]:
                before = state(env[k], int(inst.cap[k]))
                env[k, s:s + inst.dur[i]] += r[k]
                env[k] = np.maximum.accumulate(env[k][::-1])[::-1]
                after = state(env[k], int(inst.cap[k]))
                work += max(j for j in range(len(after)) if after[j] != before[j]) + 1
    return work


def earliest_fit_violations(inst, W, S):
    """For the time-indexed decoder every activity must start at the first
    t >= es_prec at which it fits beside the activities placed before it."""
    H = int(inst.dur.sum()) + 1
    use = np.zeros((inst.m, H + 1), np.int64)
    preds = {j: [] for j in range(inst.n)}
    for i, j in inst.arcs():
        preds[j].append(i)
    bad = 0
    for i in W:
        d = int(inst.dur[i])
        r = inst.req[i * inst.m:(i + 1) * inst.m]
        es = max([S[p] + inst.dur[p] for p in preds[i]], default=0)

        def fits(t):
            return all(use[k, t:t + d].max(initial=0) + r[k] <= inst.cap[k] for k in range(inst.m))
        first = next(t for t in range(es, H + 1) if fits(t))
        bad += first != S[i]
        for k in range(inst.m):
            use[k, S[i]:S[i] + d] += r[k]
    return bad


def test_decoders_on_random_lists(oracle):
    rng = np.random.default_rng(11)
    for inst in medium_instances(40):
        cp = oracle.critical_path(inst)
        for _ in range(3):
            W = random_feasible_list(inst, rng)
            for mode in (1, 2):
                cmax, S, _ = oracle.decode(inst, W, mode)
                rc, c2 = oracle.check_schedule(inst, S)
                assert rc == 0 and c2 == cmax == S[inst.n - 1]
                assert cmax >= cp
                for k in range(inst.m):
                    load = int(sum(inst.req[i * inst.m + k] * inst.dur[i] for i in range(inst.n)))
                    assert cmax >= -(-load // int(inst.cap[k]))
            _, S_t, _ = oracle.decode(inst, W, 1)
            assert earliest_fit_violations(inst, W, S_t) == 0
            c_cap, S_c, _ = oracle.decode(inst, W, 2)
            c_env, S_env = decode_by_envelope(inst, W)
            assert c_cap == c_env and S_c.tolist() == S_env.tolist()


def test_serial_sgs_leaves_no_idle_step(oracle):
    """Every step before the makespan is covered by some activity of
    positive duration, whichever evaluator decodes and whatever the list.
    (Take an idle step t and, among the activities that start after it, the
    first in list order: everything scheduled before it ends by t, so its
    predecessors do and the resources are free from t on, and the serial
    SGS would have started it by t.)  It is why no horizon below
    UB = sum d_i holds for every list, and why the makespan never exceeds UB."""
    rng = np.random.default_rng(23)
    insts = medium_instances(20, first=400) + small_instances(60, n=7, m=2, dmax=4, rmax=4, first=900)
    for inst in insts:
        ub = int(sum(inst.dur))
        for _ in range(4):
            W = random_feasible_list(inst, rng)
            for mode in (1, 2):
                cmax, S, _ = oracle.decode(inst, W, mode)
                assert cmax <= ub
                covered = np.zeros(max(cmax, 1), bool)
                for i in range(inst.n):
                    if inst.dur[i] > 0:
                        covered[S[i]:S[i] + inst.dur[i]] = True
                assert cmax == 0 or covered[:cmax].all(), (mode, np.flatnonzero(~covered[:cmax])[:5])


def test_capacity_work_counter_matches_envelopes(oracle):
    """The capacity-indexed work count (Alg. 4 loop steps) equals the one
    read off explicit usage envelopes."""
    rng = np.random.default_rng(17)
    for inst in medium_instances(16, first=230):
        for _ in range(2):
            W = random_feasible_list(inst, rng)
            assert oracle.decode(inst, W, 2)[2] == capacity_work_by_envelope(inst, W)


def test_brute_force_small(oracle):
    for inst in small_instances(25):
        opt = oracle.brute_force_starts(inst)
        t_best, t_lists = oracle.brute_force_lists(inst, 1)
        c_best, c_lists = oracle.brute_force_lists(inst, 2)
        assert t_best == opt                      # some list reaches the optimum
        assert c_best >= opt and t_lists == c_lists
        assert opt >= oracle.critical_path(inst)


def test_unlimited_capacity_gives_cpm(oracle):
    rng = np.random.default_rng(3)
    for inst in medium_instances(20):
        big = np.array([inst.req[k::inst.m].sum() + 1 for k in range(inst.m)], np.int32)
        free = Instance(inst.n, inst.m, inst.dur, big, inst.req, inst.succ_off, inst.succ)
        es = es_by_paths(free)
        W = random_feasible_list(free, rng)
        for mode in (1, 2):
            cmax, S, _ = oracle.decode(free, W, mode)
            assert S.tolist() == es and cmax == oracle.critical_path(free) == es[-1]


def test_zero_demands_give_cpm(oracle):
    for inst in medium_instances(10, first=50):
        z = Instance(inst.n, inst.m, inst.dur, inst.cap, np.zeros_like(inst.req),
                     inst.succ_off, inst.succ)
        es = es_by_paths(z)
        W = oracle.initial_order(z)
        for mode in (1, 2):
            assert oracle.decode(z, W, mode)[1].tolist() == es


def test_critical_path_by_path_enumeration(oracle):
    for inst in medium_instances(30, first=100):
        paths = all_paths(inst, 0, inst.n - 1)
        assert oracle.critical_path(inst) == max(sum(int(inst.dur[x]) for x in p[:-1]) for p in paths)


def test_time_work_counter_matches_window_scan(oracle):
    """Alg. 5 visits t = es_prec .. s+d-1, so its steps are sum(s + d - es_prec)."""
    rng = np.random.default_rng(5)
    for inst in medium_instances(10, first=200):
        W = random_feasible_list(inst, rng)
        _, S, work = oracle.decode(inst, W, 1)
        preds = {j: [] for j in range(inst.n)}
        for i, j in inst.arcs():
            preds[j].append(i)
        expect = sum(int(S[i] + inst.dur[i]) - max([int(S[p] + inst.dur[p]) for p in preds[i]], default=0)
                     for i in range(inst.n))
        assert work == expect


# ----------------------------------------------- moves, levels, initial W
def test_eq5_eq6_equal_list_feasibility(oracle):
    rng = np.random.default_rng(13)
    for inst in medium_instances(30, first=300):
        W = random_feasible_list(inst, rng)
        for u in range(1, inst.n - 2):
            for v in range(u + 1, inst.n - 1):
                Wc = W.copy()
                Wc[u], Wc[v] = W[v], W[u]
                assert oracle.move_feasible(inst, W, u, v) == list_is_feasible(inst, Wc)


def test_levels_and_initial_order(oracle):
    for inst in medium_instances(20, first=400):
        lev = oracle.levels(inst)
        for j in range(inst.n):
            assert lev[j] == max(len(p) - 1 for p in all_paths(inst, 0, j))
        W = oracle.initial_order(inst)
        assert list_is_feasible(inst, W)
        assert [(lev[i], i) for i in W] == sorted((lev[i], i) for i in range(inst.n))
        key = np.random.default_rng(1).integers(0, 5, inst.n).astype(np.int32)
        Wk = oracle.initial_order(inst, key)
        assert [(lev[i], key[i], i) for i in Wk] == sorted((lev[i], key[i], i) for i in range(inst.n))
        assert Wk[0] == 0 and Wk[-1] == inst.n - 1


# ------------------------------------------------------------ tabu search
def replay(oracle, inst, res, delta, mode):
    """Checks a trace against list feasibility and the decoder, and
    re-counts the feasible neighbours of every visited list."""
    W = oracle.initial_order(inst)
    C0 = oracle.decode(inst, W, mode)[0]
    best = C0
    evaluated = 0
    for u, v, c in res["trace"]:
        evaluated += sum(1 for a in range(1, inst.n - 1) for b in range(a + 1, min(a + delta, inst.n - 2) + 1)
                         if list_is_feasible(inst, np.r_[W[:a], W[b], W[a + 1:b], W[a], W[b + 1:]]))
        if (u, v) != (0, 0):
            W = W.copy()
            W[u], W[v] = W[v], W[u]
            assert list_is_feasible(inst, W)
            assert oracle.decode(inst, W, mode)[0] == c
            best = min(best, c)
    assert evaluated == res["evaluated"]
    assert best == res["best_cmax"]


@pytest.mark.parametrize("mode", [1, 2])
def test_tabu_trace_is_consistent(oracle, mode):
    for inst in medium_instances(6, first=500):
        res = oracle.tabu_search(inst, 30, 6, 7, mode, 0, trace=True)
        assert res["status"] == 0 and res["iterations"] == 30
        replay(oracle, inst, res, 6, mode)
        rc, cm = oracle.check_schedule(inst, res["best_S"])
        assert rc == 0 and cm == res["best_cmax"]


def test_tabu_stops_at_critical_path(oracle):
    inst = medium_instances(1, first=600)[0]
    big = np.array([inst.req[k::inst.m].sum() + 1 for k in range(inst.m)], np.int32)
    free = Instance(inst.n, inst.m, inst.dur, big, inst.req, inst.succ_off, inst.succ)
    res = oracle.tabu_search(free, 50, 10, 10, 1, 1)
    assert res["iterations"] == 0 and res["evaluated"] == 0
    assert res["best_cmax"] == res["cp"]


def test_chain_has_empty_neighbourhood(oracle):
    n = 6
    succ_sets = [[1]] + [[i + 1] for i in range(1, n + 1)] + [[]]
    off = np.r_[0, np.cumsum([len(s) for s in succ_sets])].astype(np.int32)
    chain = Instance(n + 2, 1, np.r_[0, np.ones(n, np.int32) * 2, 0].astype(np.int32),
                     np.array([1], np.int32), np.r_[0, np.ones(n), 0].astype(np.int32),
                     off, np.array([x for s in succ_sets for x in s], np.int32))
    res = oracle.tabu_search(chain, 5, 4, 3, 1, 0, trace=True)
    assert res["evaluated"] == 0 and res["iterations"] == 5
    assert (res["trace"][:, :2] == 0).all() and res["best_cmax"] == 2 * n


def test_batch_equals_single(oracle):
    insts = medium_instances(8, first=700)
    params = [(20, 8, 9, 0, 1)] * len(insts)
    batch = oracle.tabu_search_batch(insts, params, 4)
    for inst, b in zip(insts, batch):
        s = oracle.tabu_search(inst, 20, 8, 9, 0, 1)
        assert b["best_cmax"] == s["best_cmax"] and b["evaluated"] == s["evaluated"]
        assert b["best_W"].tolist() == s["best_W"].tolist()


# ------------------------------------- tabu search: restated from the paper
def sgs_earliest_fit(inst, W):
    """Serial SGS (Alg. 7) from its definition: in list order, each
    activity starts at the first t >= its predecessors' latest finish at
    which its demand fits beside everything placed before it."""
    H = int(inst.dur.sum()) + 1
    use = np.zeros((inst.m, H + 1), np.int64)
    preds = {j: [] for j in range(inst.n)}
    for i, j in inst.arcs():
        preds[j].append(i)
    S = np.zeros(inst.n, np.int64)
    for i in W:
        d = int(inst.dur[i])
        r = inst.req[i * inst.m:(i + 1) * inst.m]
        es = max([S[p] + inst.dur[p] for p in preds[i]], default=0)
        S[i] = next(t for t in range(es, H + 1)
                    if all(use[k, t:t + d].max(initial=0) + r[k] <= inst.cap[k] for k in range(inst.m)))
        for k in range(inst.m):
            use[k, S[i]:S[i] + d] += r[k]
    return int(max(S + inst.dur)), S


def level_order(inst, key=None):
    """W0 of Sec. 4.1: ascending (level, key, label), level = most arcs on
    a path from the source, by path enumeration; key = 0 unless shuffle
    keys are given."""
    lev = [max(len(p) - 1 for p in all_paths(inst, 0, j)) for j in range(inst.n)]
    kk = [0] * inst.n if key is None else [int(x) for x in key]
    return np.array(sorted(range(inst.n), key=lambda j: (lev[j], kk[j], j)), np.int32)


def is_tabu(history, x, L):
    """The simple tabu list of Alg. 3 stated over the history of applied
    moves m_0, m_1, ...: each iteration writes its move into the cache and
    evicts the move of L iterations before, clearing its cache entry even
    when a later copy of the same move is still listed.  So x is tabu iff
    its last occurrence i is one of the last L moves and no earlier copy of
    x was evicted after i, i.e. none lies in (i - L, j - L], j the last
    iteration."""
    j = len(history) - 1
    last = max((i for i, m in enumerate(history) if m == x), default=None)
    if last is None or last <= j - L:
        return False
    return not any(history[k] == x for k in range(max(0, last - L + 1), j - L + 1))


def tabu_search_restated(inst, iterations, delta, L, mode, stop_at_cp):
    """Sec. 6 iteration by definitions: every swap (u, v), 1 <= u < v <=
    N-2, v - u <= delta, whose swapped list is precedence-feasible is
    decoded; a tabu move is admissible only if strictly better than the best
    so far; the admissible move with the smallest (C, u, v) is applied; with
    none, the list stays and the empty move enters the tabu list."""
    decode = (lambda x, w: sgs_earliest_fit(x, w)[0]) if mode == 1 else (lambda x, w: decode_by_envelope(x, w)[0])
    cp = max(sum(int(inst.dur[x]) for x in p[:-1]) for p in all_paths(inst, 0, inst.n - 1))
    W = level_order(inst)
    best, best_W = decode(inst, W), W.copy()
    history, trace, evaluated = [], [], 0
    for _ in range(iterations):
        if stop_at_cp and best == cp:
            break
        cands = []
        for u in range(1, inst.n - 2):
            for v in range(u + 1, min(u + delta, inst.n - 2) + 1):
                Wc = W.copy()
                Wc[u], Wc[v] = W[v], W[u]
                if not list_is_feasible(inst, Wc):
                    continue
                c = decode(inst, Wc)
                evaluated += 1
                if not is_tabu(history, (u, v), L) or c < best:
                    cands.append((c, u, v))
        if cands:
            c, u, v = min(cands)
            W[u], W[v] = W[v], W[u]
            if c < best:
                best, best_W = c, W.copy()
        else:
            u = v = 0
            c = trace[-1][2] if trace else decode(inst, W)
        history.append((u, v))
        trace.append((u, v, c))
    return dict(trace=trace, evaluated=evaluated, best_cmax=best, best_W=best_W)


def restatement_cases():
    """Tiny instances, plus three found by search on which a tabu move is
    taken again by aspiration while its older copy is still listed (the
    case reading R7 decides)."""
    out = [(x, d, L, stop) for x in small_instances(12, n=6, first=40)
           for d, L, stop in ((1, 1, 0), (2, 2, 0), (3, 3, 1), (x.n, 5, 0), (2, 9, 0))]
    for s, d, L in ((264, 3, 5), (308, 4, 12), (170, 4, 12)):
        out.append((generate(s, 6 + s % 9, 1 + s % 3, 150 + 30 * (s % 3), 20 + 30 * (s % 3), dmax=3 + s % 6,
                             rmax=2 + s % 7, relabel=bool(s % 2), stream=97), d, L, 0))
    return out


def restatement_mismatches(oracle, mode, iterations=40):
    """Runs whose oracle trajectory differs from the restatement, and how
    many empty moves and aspirated repeats of a listed move the
    restatement made."""
    bad = empty = dup = 0
    for inst, delta, L, stop in restatement_cases():
        ref = tabu_search_restated(inst, iterations, delta, L, mode, stop)
        got = oracle.tabu_search(inst, iterations, delta, L, mode, stop, trace=True)
        same = ([tuple(int(x) for x in t) for t in got["trace"][:got["iterations"]]] == ref["trace"]
                and got["evaluated"] == ref["evaluated"] and got["best_cmax"] == ref["best_cmax"]
                and got["best_W"].tolist() == ref["best_W"].tolist())
        bad += not same
        moves = [t[:2] for t in ref["trace"]]
        empty += moves.count((0, 0))
        dup += sum(1 for i, m in enumerate(moves) if m != (0, 0) and m in moves[max(0, i - L):i])
    return bad, empty, dup


@pytest.mark.parametrize("mode", [1, 2])
def test_tabu_search_equals_restatement(oracle, mode):
    """The oracle's whole trajectory -- every selected move, its makespan,
    the neighbour count and the best list -- equals the search restated
    from the definitions, with tabu lists short enough that entries are
    evicted, leave no admissible move, and are taken again by aspiration."""
    bad, empty, dup = restatement_mismatches(oracle, mode)
    assert bad == 0
    assert empty > 0 and dup > 0


# ------------------------------------------------- evaluator selection (R8)
def chain_instance(durs, cap):
    """Source, the activities in one chain, sink; one resource."""
    n = len(durs)
    succ_sets = [[1]] + [[i + 2] for i in range(n)] + [[]]
    off = np.r_[0, np.cumsum([len(s) for s in succ_sets])].astype(np.int32)
    return Instance(n + 2, 1, np.r_[0, durs, 0].astype(np.int32), np.array([cap], np.int32),
                    np.r_[0, np.ones(n), 0].astype(np.int32), off,
                    np.array([x for s in succ_sets for x in s], np.int32))


def test_selection_rule(oracle):
    """Capacity-indexed exactly when CP * M > 12 * sum R_k (reading R8), the
    critical path taken by path enumeration; equality stays time-indexed."""
    long_low = [generate(s, 10 + s % 5, 1 + s % 2, 210, 10, dmax=50, rmax=2, stream=96) for s in range(30)]
    seen = set()
    for inst in medium_instances(30, first=1200) + long_low:
        cp = max(sum(int(inst.dur[x]) for x in p[:-1]) for p in all_paths(inst, 0, inst.n - 1))
        want = 2 if cp * inst.m > 12 * int(inst.cap.sum()) else 1
        assert oracle.select_mode(inst) == want
        seen.add(want)
    assert seen == {1, 2}
    for R in (1, 2, 5):
        assert oracle.select_mode(chain_instance([6 * R, 6 * R], R)) == 1            # CP = 12 R
        assert oracle.select_mode(chain_instance([6 * R, 6 * R + 1], R)) == 2        # CP = 12 R + 1


# ------------------------------------------------- checker: negative cases
def test_checker_rejects_violations(oracle):
    """Eqs. 3-4 with their boundaries: a successor may start exactly at its
    predecessor's finish, one step earlier is a precedence violation; an
    activity may start where another with the full capacity ends (intervals
    are half-open), one step of overlap overloads; negative starts are
    refused."""
    inst, vals = table1()
    W = np.array(vals["W"], np.int32)
    S = oracle.decode(inst, W, 1)[1].astype(np.int32)
    assert oracle.check_schedule(inst, S)[0] == 0
    tight = [(i, j) for i, j in inst.arcs() if S[j] == S[i] + inst.dur[i] and S[j] > 0 and inst.dur[i] > 0]
    assert tight
    for i, j in tight:
        bad = S.copy()
        bad[j] -= 1
        assert oracle.check_schedule(inst, bad)[0] == 1
    neg = S.copy()
    neg[0] = -1
    assert oracle.check_schedule(inst, neg)[0] == 3
    # two unrelated activities that each take the whole capacity
    succ_sets = [[1, 2], [3], [3], []]
    off = np.r_[0, np.cumsum([len(s) for s in succ_sets])].astype(np.int32)
    two = Instance(4, 1, np.array([0, 2, 3, 0], np.int32), np.array([4], np.int32),
                   np.array([0, 4, 4, 0], np.int32), off, np.array([x for s in succ_sets for x in s], np.int32))
    assert oracle.check_schedule(two, np.array([0, 0, 2, 5], np.int32)) == (0, 5)
    assert oracle.check_schedule(two, np.array([0, 0, 1, 4], np.int32))[0] == 2
    assert oracle.check_schedule(two, np.array([0, 0, 2, 4], np.int32))[0] == 1      # sink before b ends
