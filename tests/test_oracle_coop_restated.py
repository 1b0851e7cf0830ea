"""The co-operative search of the CPU reference against a restatement.

The searches of Sec. 6.1 are restated here from the paper and the readings
C1-C8 and F1-F3, with data structures of their own: schedules by earliest
fit or explicit envelopes, feasibility of every swapped list checked
directly, the tabu list as the history of applied moves, the backward pass
of FBI on an explicitly reversed instance, and Eq. 8 with the mathematical
exponential.  On tiny instances the reference's result -- best list and
makespan, evaluated neighbours, iterations -- must equal the restatement's,
over runs that write, time out, diversify and improve slots by FBI.  CPU
only.
"""
import math

import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300.instances import Instance

from test_oracle_pins import (all_paths, decode_by_envelope, is_tabu, level_order, list_is_feasible,
                              medium_instances, sgs_earliest_fit, small_instances)


def decoder(mode):
    return sgs_earliest_fit if mode == 1 else decode_by_envelope


def reversed_instance(inst):
    """Every arc turned around: successors act as predecessors."""
    succ = [[] for _ in range(inst.n)]
    for i, j in inst.arcs():
        succ[j].append(i)
    off = np.r_[0, np.cumsum([len(x) for x in succ])].astype(np.int32)
    flat = np.array([x for xs in succ for x in xs], np.int32)
    return Instance(inst.n, inst.m, inst.dur, inst.cap, inst.req, off, flat)


def fbi_restated(inst, W, mode):
    """F1-F3: right-justify on the reversed network in order of falling
    finish time, mirror, take the activities in order of rising mirrored
    start as the new list; repeat while the makespan falls strictly."""
    dec, rev = decoder(mode), reversed_instance(inst)
    d = inst.dur.astype(np.int64)
    W = [int(a) for a in W]
    C, S = dec(inst, W)
    while True:
        pos = {a: p for p, a in enumerate(W)}
        Wb = sorted(W, key=lambda a: (-(S[a] + d[a]), -pos[a]))
        T, tau = dec(rev, Wb)
        mirrored = {a: T - tau[a] - d[a] for a in W}
        Wn = sorted(W, key=lambda a: (mirrored[a], pos[a]))
        C2, S2 = dec(inst, Wn)
        if not C2 < C:
            return np.array(W, np.int32)
        W, C, S = Wn, C2, S2


def feasible_swaps(inst, W, delta):
    out = []
    for u in range(1, inst.n - 2):
        for v in range(u + 1, min(u + delta, inst.n - 2) + 1):
            Wc = W.copy()
            Wc[u], Wc[v] = W[v], W[u]
            if list_is_feasible(inst, Wc):
                out.append((u, v))
    return out


def eq8(c_k, c_star, ic_k, i_block):
    """Eq. 8 with the quantity factor read as I_block / 5 (reading C6)."""
    q = math.exp(-100.0 * (c_k / c_star - 1.0)) if c_star > 0 else 1.0
    return int(math.floor(i_block / 5.0 * (0.8 * q + 0.2 * math.exp(-4.0 * ic_k / i_block))))


def coop_restated(inst, iterations, delta, L, mode, stop, B, F, phi_max, phi_steps, assign_fixed, keys, words,
                  fbi_every):
    dec = decoder(mode)
    cmax = (lambda W: dec(inst, W)[0])
    cp = max(sum(int(inst.dur[x]) for x in p[:-1]) for p in all_paths(inst, 0, inst.n - 1))
    ev = dict(writes=0, timeouts=0, diversified=0, fbi=0)
    # C7: the working set
    slots = []
    for k in range(F):
        W = level_order(inst, None if keys is None else keys[k])
        if fbi_every > 0 and k % fbi_every == fbi_every - 1:
            W2 = fbi_restated(inst, W, mode)
            ev["fbi"] += W2.tolist() != W.tolist()
            W = W2
        slots.append(dict(W=W, hist=[], C=cmax(W), phi=0, IC=0))
    blocks = [dict(cursor=0) for _ in range(B)]
    pointer = [0]
    evaluated = [0]

    def best_known():                                   # C2
        return min([s["C"] for s in slots] + [b["Cbb"] for b in blocks if "Cbb" in b])

    def read(b, c_star):                                # C5
        x, k = blocks[b], pointer[0]
        pointer[0] = (k + 1) % F
        f = slots[k]
        f["phi"] += 1
        x.update(W=f["W"].copy(), hist=list(f["hist"]), slot=k, Cread=f["C"], ICread=f["IC"], since=0)
        x["C"] = f["C"]
        if f["phi"] > phi_max and phi_steps > 0:
            for _ in range(phi_steps):
                moves = feasible_swaps(inst, x["W"], delta)
                if not moves:
                    break
                w = int(words[b][x["cursor"] % len(words[b])])
                x["cursor"] += 1
                u, v = moves[(w * len(moves)) >> 32]
                x["W"][u], x["W"][v] = x["W"][v], x["W"][u]
            x["C"] = cmax(x["W"])
            ev["diversified"] += 1
        x["Cbb"], x["Wbb"] = x["C"], x["W"].copy()
        x["assigned"] = assign_fixed if assign_fixed > 0 else eq8(f["C"], c_star, f["IC"], iterations)

    c0 = best_known()
    for b in range(B):
        read(b, c0)
    its = 0
    while its < iterations:
        c_star = best_known()
        if stop and c_star == cp:                       # C8
            break
        for x in blocks:                                # C1: one Sec. 6 iteration each
            cands = []
            for u, v in feasible_swaps(inst, x["W"], delta):
                Wc = x["W"].copy()
                Wc[u], Wc[v] = Wc[v], Wc[u]
                c = cmax(Wc)
                evaluated[0] += 1
                if not is_tabu(x["hist"], (u, v), L) or c < c_star:
                    cands.append((c, u, v))
            if cands:
                c, u, v = min(cands)
                x["W"][u], x["W"][v] = x["W"][v], x["W"][u]
                x["C"] = c
            else:
                u = v = 0
            x["hist"].append((u, v))
            if x["C"] < x["Cbb"]:
                x["Cbb"], x["Wbb"] = x["C"], x["W"].copy()
            x["since"] += 1
        its += 1
        exchange = []
        for x in blocks:                                # C3, C4: writes in block order
            improved = x["Cbb"] < x["Cread"]
            exchange.append(improved or x["since"] > x["assigned"])
            if not exchange[-1]:
                continue
            ev["timeouts"] += not improved
            f = slots[x["slot"]]
            if improved and x["Cbb"] < f["C"]:
                f.update(W=x["Wbb"].copy(), hist=list(x["hist"]), C=x["Cbb"], IC=x["ICread"] + x["since"], phi=0)
                ev["writes"] += 1
            else:
                f["IC"] += x["since"]
        if its < iterations:
            c_star = best_known()
            for b in range(B):                          # C5: reads in block order
                if exchange[b]:
                    read(b, c_star)
    best = min(range(F), key=lambda k: (slots[k]["C"], k))
    C, W = slots[best]["C"], slots[best]["W"]
    for x in blocks:                                    # C8
        if x["Cbb"] < C:
            C, W = x["Cbb"], x["Wbb"]
    return dict(best_cmax=C, best_W=W, evaluated=evaluated[0], iterations=its * B, events=ev)


def cases():
    out = []
    for k, inst in enumerate(small_instances(6, n=7, first=60) + medium_instances(8, first=900)):
        if inst.n > 12:
            continue
        B, F = 1 + k % 3, 1 + (k * 5) % 4
        out.append((inst, dict(iterations=24, delta=2 + k % 3, L=2 + k % 4, stop=k % 2, B=B, F=F,
                               phi_max=k % 3, phi_steps=2 + k % 3, assign_fixed=0 if k % 4 else 3,
                               fbi_every=(0, 1, 2)[k % 3], seed=7 + k)))
    # instances on which blocks improve what they read and write it back
    pool = medium_instances(40, first=900)
    for k in (4, 9, 21, 26, 38):
        out.append((pool[k], dict(iterations=30, delta=3, L=3, stop=0, B=2 + k % 2, F=2 + k % 3, phi_max=1,
                                  phi_steps=2, assign_fixed=0, fbi_every=2, seed=7 + k)))
    return out


def coop_mismatches(oracle, mode):
    """Cases whose reference result differs from the restatement, and the
    events the restatement went through."""
    bad, seen = 0, dict(writes=0, timeouts=0, diversified=0, fbi=0)
    for inst, c in cases():
        keys, words = I.coop_inputs(inst, c["seed"], c["F"], c["B"], 16)
        ref = coop_restated(inst, c["iterations"], c["delta"], c["L"], mode, c["stop"], c["B"], c["F"],
                            c["phi_max"], c["phi_steps"], c["assign_fixed"], keys, words, c["fbi_every"])
        got = oracle.coop_search(inst, c["iterations"], c["delta"], c["L"], mode, c["stop"], c["B"], c["F"],
                                 c["phi_max"], c["phi_steps"], c["assign_fixed"], keys, words,
                                 fbi_every=c["fbi_every"])
        bad += not (got["status"] == 0 and got["best_cmax"] == ref["best_cmax"]
                    and got["evaluated"] == ref["evaluated"] and got["iterations"] == ref["iterations"]
                    and got["best_W"].tolist() == [int(a) for a in ref["best_W"]])
        for k in seen:
            seen[k] += ref["events"][k]
    return bad, seen


@pytest.mark.parametrize("mode", [1, 2])
def test_cooperation_equals_restatement(oracle, mode):
    bad, seen = coop_mismatches(oracle, mode)
    assert bad == 0
    assert all(v > 0 for v in seen.values()), seen


@pytest.mark.parametrize("mode", [1, 2])
def test_fbi_equals_restatement(oracle, mode):
    changed = 0
    for inst in small_instances(10, n=7, first=80) + [x for x in medium_instances(12, first=950) if x.n <= 16]:
        for key_seed in (None, 3, 4):
            key = None if key_seed is None else I.level_keys(inst, key_seed)
            W = level_order(inst, key)
            got, c, _ = oracle.fbi(inst, W, mode)
            assert got.tolist() == fbi_restated(inst, W, mode).tolist()
            changed += got.tolist() != W.tolist()
    assert changed > 0
