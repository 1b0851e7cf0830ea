"""Test-only instance family whose precedence graphs have arcs that skip
layers (seeded inputs; no search arithmetic).

The workload generator draws layered graphs whose arcs join adjacent layers
only.  Real projects also have arcs from an activity to one several levels
later, as the Table 1 example does (3 -> 10, 1 -> 6).  This family starts
from a layered instance, adds arcs a -> b between non-dummy activities whose
levels differ by two or more when b is not already reachable from a, then
removes every arc implied by a longer path (transitive reduction) and
reconnects the dummies, so the result is again a valid instance of Sec. 2:
acyclic, 0 the only activity without a predecessor, N-1 the only one
without a successor, every arc necessary.  Labels can be permuted so that
they are not a topological order.
"""
from __future__ import annotations

from typing import List

import numpy as np

from paper_1711_04556_gb300 import instances as I


def _levels(n, succ):
    """Longest unit-weight path from activity 0 (Kahn order)."""
    indeg = [0] * n
    for a in range(n):
        for b in succ[a]:
            indeg[b] += 1
    order, stack = [], [a for a in range(n) if indeg[a] == 0]
    while stack:
        a = stack.pop()
        order.append(a)
        for b in succ[a]:
            indeg[b] -= 1
            if indeg[b] == 0:
                stack.append(b)
    lev = [0] * n
    for a in order:
        for b in succ[a]:
            lev[b] = max(lev[b], lev[a] + 1)
    return lev


def reachable(succ, a, b, skip_arc=None):
    """b reachable from a, optionally without using the arc skip_arc."""
    stack, seen = [a], {a}
    while stack:
        x = stack.pop()
        for y in succ[x]:
            if (x, y) == skip_arc:
                continue
            if y == b:
                return True
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return False


def transitive_reduction(succ):
    n = len(succ)
    for a in range(n):
        for b in sorted(succ[a]):
            if reachable(succ, a, b, skip_arc=(a, b)):
                succ[a].discard(b)
    return succ


def with_skip_arcs(seed: int, n: int = 30, m: int = 4, nc100: int = 150, rs100: int = 50, extra: int = 12,
                   relabel: bool = False, **kw) -> I.Instance:
    base = I.generate(seed, n, m, nc100, rs100, stream=41, **kw)
    N = base.n
    succ = [set(int(x) for x in base.successors(i)) for i in range(N)]
    lev = _levels(N, succ)
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x5C1B]))
    added, tries = 0, 0
    while added < extra and tries < 50 * extra:
        tries += 1
        a, b = (int(x) for x in rng.integers(1, N - 1, 2))
        if lev[b] < lev[a] + 2 or b in succ[a] or reachable(succ, a, b):
            continue
        succ[a].add(b)
        added += 1
    # dummies: the source precedes exactly the activities without another
    # predecessor, the sink follows those without another successor
    succ[0] = set(range(1, N - 1))
    for i in range(1, N - 1):
        succ[i].add(N - 1)
    succ = transitive_reduction(succ)
    dur, req = base.dur.copy(), base.req.reshape(N, m).copy()
    if relabel:
        perm = np.arange(N)
        perm[1:N - 1] = 1 + rng.permutation(N - 2)       # old label -> new label
        inv = np.argsort(perm)
        dur, req = dur[inv], req[inv]
        succ = [{int(perm[j]) for j in succ[int(inv[i])]} for i in range(N)]
    off = np.zeros(N + 1, np.int32)
    off[1:] = np.cumsum([len(s) for s in succ])
    arcs = np.array([x for s in succ for x in sorted(s)], np.int32)
    return I.Instance(N, m, dur, base.cap.copy(), req.reshape(-1).astype(np.int32), off, arcs,
                      dict(base.meta, skip_arcs=added, relabel=relabel))


def skip_arc_batch(count: int, n: int = 30, first: int = 0, **kw) -> List[I.Instance]:
    return [with_skip_arcs(s, n, 4, I.NC_GRID[s % 3], I.RS_GRID4[(s // 3) % 4], relabel=bool(s % 2), **kw)
            for s in range(first, first + count)]
