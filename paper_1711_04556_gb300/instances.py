"""Seeded synthetic RCPSP instances (inputs only; none of the search arithmetic).

The paper measures on PSPLIB J30-J120 and on ProGen-generated sets (Sec. 7,
Sec. 7.1).  Neither is available here, so every workload is drawn by this
module from a seed.  The recipe mirrors the ProGen parameters the paper names
(number of activities, resources, network complexity NC, resource strength
RS) and the problem statement of Sec. 2:

* activities 0 and N-1 are dummies with zero duration and zero demand;
* durations are uniform integers in [dmin, dmax];
* each (activity, resource) pair is used with probability ``p_use``; a used
  pair draws a demand uniform in [1, rmax];
* the precedence graph is layered: non-dummy activities get a layer, every
  activity past the first layer gets one predecessor in the layer before,
  every activity before the last layer gets one successor in the layer after,
  and extra arcs between adjacent layers are drawn until the non-dummy arc
  count reaches round(NC * n).  An arc between adjacent layers can never be
  implied by a longer path, so the graph is transitively reduced by
  construction.  The source precedes every activity without a predecessor and
  the sink follows every activity without a successor;
* the capacity of resource k is K_min + round_half_up(RS * (K_max - K_min)),
  K_min the largest single demand, K_max the peak of the demand profile of
  the earliest-start (infinite capacity) schedule; an unused resource gets
  capacity 1.

This module is shared by the tests, the benchmark and the CPU reference: it
makes inputs and never computes a schedule evaluation, a move or a search
step.
"""
from __future__ import annotations

import dataclasses
import hashlib
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Instance", "generate", "table1_instance", "config_batch", "level_keys",
    "NC_GRID", "RS_GRID4", "RS_GRID5",
]

NC_GRID = (150, 180, 210)              # network complexity in hundredths
RS_GRID4 = (20, 50, 70, 100)           # resource strength in hundredths
RS_GRID5 = (10, 20, 50, 70, 100)


@dataclasses.dataclass
class Instance:
    """One RCPSP instance in the layout of the C boundary (all int32).

    n        -- number of activities N, dummies 0 and N-1 included
    m        -- number of renewable resources M
    dur      -- [N] durations, dur[0] = dur[N-1] = 0
    cap      -- [M] capacities R_k >= 1
    req      -- [N*M] demands r_{i,k}, row-major by activity
    succ_off -- [N+1] CSR offsets into succ
    succ     -- [|E|] successor lists
    """
    n: int
    m: int
    dur: np.ndarray
    cap: np.ndarray
    req: np.ndarray
    succ_off: np.ndarray
    succ: np.ndarray
    meta: dict = dataclasses.field(default_factory=dict)

    def successors(self, i: int) -> np.ndarray:
        return self.succ[self.succ_off[i]:self.succ_off[i + 1]]

    def arcs(self) -> List[tuple]:
        return [(i, int(j)) for i in range(self.n) for j in self.successors(i)]

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (np.array([self.n, self.m], np.int32), self.dur, self.cap,
                  self.req, self.succ_off, self.succ):
            h.update(np.ascontiguousarray(a, np.int32).tobytes())
        return h.hexdigest()[:16]

    def to_text(self) -> str:
        """Plain text form: header, then one line per activity."""
        lines = [f"{self.n} {self.m}", " ".join(str(int(c)) for c in self.cap)]
        for i in range(self.n):
            s = self.successors(i)
            lines.append(" ".join(
                [str(int(self.dur[i]))]
                + [str(int(x)) for x in self.req[i * self.m:(i + 1) * self.m]]
                + [str(len(s))] + [str(int(x)) for x in s]))
        return "\n".join(lines) + "\n"

    @staticmethod
    def from_text(text: str, meta: Optional[dict] = None) -> "Instance":
        rows = [r.split() for r in text.strip().splitlines()
                if r.strip() and not r.lstrip().startswith("#")]
        n, m = int(rows[0][0]), int(rows[0][1])
        cap = np.array([int(x) for x in rows[1]], np.int32)
        dur = np.zeros(n, np.int32)
        req = np.zeros(n * m, np.int32)
        succ_lists = []
        for i in range(n):
            r = [int(x) for x in rows[2 + i]]
            dur[i] = r[0]
            req[i * m:(i + 1) * m] = r[1:1 + m]
            k = r[1 + m]
            succ_lists.append(r[2 + m:2 + m + k])
        off = np.zeros(n + 1, np.int32)
        off[1:] = np.cumsum([len(s) for s in succ_lists])
        succ = np.array([x for s in succ_lists for x in s], np.int32)
        return Instance(n, m, dur, cap, req, off, succ, dict(meta or {}))


def _csr(n: int, succ_sets: Sequence[Sequence[int]]):
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum([len(s) for s in succ_sets])
    succ = np.array([x for s in succ_sets for x in sorted(s)], np.int32)
    return off, succ


def _earliest_starts(n: int, dur: np.ndarray, succ_sets, topo: Sequence[int]):
    """Infinite-capacity earliest starts, used only to size capacities."""
    es = np.zeros(n, np.int64)
    for i in topo:
        for j in succ_sets[i]:
            es[j] = max(es[j], es[i] + dur[i])
    return es


def generate(seed: int, n: int = 30, m: int = 4, nc100: int = 150, rs100: int = 50,
             dmin: int = 1, dmax: int = 10, rmax: int = 10, p_use: float = 0.5,
             relabel: bool = False, stream: int = 0) -> Instance:
    """Draw one instance with ``n`` non-dummy activities (N = n + 2).

    ``nc100`` and ``rs100`` are NC and RS in hundredths so that the arc
    target and the capacities are exact integers.  ``stream`` separates
    generator families that share seeds (the batch configurations).
    ``relabel`` permutes the non-dummy labels so that labels are not a
    topological order.
    """
    if n < 1 or m < 1:
        raise ValueError("need n >= 1 and m >= 1")
    rng = np.random.Generator(np.random.Philox(key=[seed, stream]))
    N = n + 2
    dur = np.zeros(N, np.int32)
    dur[1:N - 1] = rng.integers(dmin, dmax + 1, n)
    req = np.zeros((N, m), np.int32)
    use = rng.random((n, m)) < p_use
    val = rng.integers(1, rmax + 1, (n, m))
    req[1:N - 1] = np.where(use, val, 0)

    # ---- layered precedence graph on labels 1..n (topological labels) ----
    target = (nc100 * n + 50) // 100
    width = max(3.0, 2.0 * nc100 / 100.0 + 1.0)
    n_layers = max(1, min(n, int(round(n / width))))
    for _attempt in range(64):
        lay = np.sort(rng.integers(0, n_layers, n))
        _, lay = np.unique(lay, return_inverse=True)     # drop empty layers
        sizes = np.bincount(lay)
        room = int(np.sum(sizes[:-1] * sizes[1:]))
        if room >= target or n_layers == 1:
            break
        n_layers = max(1, n_layers - 1)
    members = [list(np.nonzero(lay == l)[0] + 1) for l in range(len(sizes))]
    succ_sets = [set() for _ in range(N)]
    pred_cnt = np.zeros(N, np.int64)
    arcs = 0

    def add(a: int, b: int) -> bool:
        nonlocal arcs
        if b in succ_sets[a]:
            return False
        succ_sets[a].add(b)
        pred_cnt[b] += 1
        arcs += 1
        return True

    for l in range(1, len(members)):
        prev = members[l - 1]
        for b in members[l]:
            add(int(prev[rng.integers(0, len(prev))]), int(b))
    for l in range(len(members) - 1):
        nxt = members[l + 1]
        for a in members[l]:
            if not succ_sets[a]:
                add(int(a), int(nxt[rng.integers(0, len(nxt))]))
    free = [(int(a), int(b)) for l in range(len(members) - 1)
            for a in members[l] for b in members[l + 1] if b not in succ_sets[a]]
    if arcs < target and free:
        pick = rng.permutation(len(free))[:target - arcs]
        for p in pick:
            add(*free[p])
    for i in range(1, N - 1):
        if pred_cnt[i] == 0:
            add(0, i)
        if not succ_sets[i]:
            add(i, N - 1)

    # ---- capacities from the earliest-start demand profile ----
    topo = list(range(N))
    es = _earliest_starts(N, dur, succ_sets, topo)
    horizon = int(np.max(es + dur)) + 1
    cap = np.ones(m, np.int32)
    for k in range(m):
        kmin = int(req[:, k].max())
        if kmin == 0:
            continue
        prof = np.zeros(horizon + 1, np.int64)
        for i in range(N):
            if req[i, k] and dur[i]:
                prof[es[i]] += req[i, k]
                prof[es[i] + dur[i]] -= req[i, k]
        kmax = int(np.cumsum(prof).max())
        cap[k] = kmin + (rs100 * (kmax - kmin) + 50) // 100

    if relabel and n > 1:
        perm = np.arange(N)
        perm[1:N - 1] = 1 + rng.permutation(n)        # old label -> new label
        inv = np.argsort(perm)
        dur = dur[inv]
        req = req[inv]
        succ_sets = [{int(perm[j]) for j in succ_sets[int(inv[i])]} for i in range(N)]
    off, succ = _csr(N, succ_sets)
    meta = dict(seed=seed, stream=stream, n_nondummy=n, nc100=nc100, rs100=rs100,
                dmin=dmin, dmax=dmax, rmax=rmax, relabel=relabel)
    return Instance(N, m, dur, cap, req.reshape(-1).astype(np.int32), off, succ, meta)


def table1_instance(cap=(6, 6)) -> Instance:
    """The 12-activity, 2-resource example of Table 1 (Sec. 2.2).

    The text gives both resources a maximal capacity of 6; ``cap`` lets the
    tests perturb it.
    """
    rows = [  # d, r0, r1, successors
        (0, 0, 0, [1, 2]), (4, 5, 3, [3, 6]), (3, 2, 1, [4, 5]), (5, 3, 2, [5, 10]),
        (5, 2, 3, [7]), (3, 3, 4, [8, 9]), (2, 4, 1, [7, 9]), (4, 2, 2, [8, 10]),
        (2, 4, 5, [11]), (3, 1, 2, [11]), (4, 2, 2, [11]), (0, 0, 0, []),
    ]
    N, m = len(rows), 2
    dur = np.array([r[0] for r in rows], np.int32)
    req = np.array([[r[1], r[2]] for r in rows], np.int32).reshape(-1)
    off, succ = _csr(N, [r[3] for r in rows])
    return Instance(N, m, dur, np.array(cap, np.int32), req, off, succ,
                    dict(name="table1", cap=tuple(cap)))


def level_keys(inst: Instance, seed: int) -> np.ndarray:
    """Random tie-break keys for shuffling activities within a level (Sec. 4.1).

    The initial order groups activities by level; alternative initial orders
    come from shuffling each level.  The shuffle is expressed as one random
    key per activity (ties broken by label), drawn here and passed to both
    the CUDA path and the CPU reference as an input.
    """
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x5EED]))
    return rng.integers(0, 2**31 - 1, inst.n).astype(np.int32)


def coop_inputs(inst: Instance, seed: int, working_set: int, blocks: int, words_per_block: int):
    """Inputs of a co-operative search (Sec. 6.1): the shuffle keys of the
    working set's initial lists (slot 0 keeps the unshuffled level order,
    slot k >= 1 uses level_keys(inst, seed + k)) and the random words the
    blocks draw their diversification swaps from, [blocks, words_per_block]
    uint32.  Drawn here and passed to both the CUDA path and the CPU
    reference as inputs."""
    keys = [None] + [level_keys(inst, seed + k) for k in range(1, working_set)]
    rng = np.random.Generator(np.random.Philox(key=[seed, 0xD1CE]))
    words = rng.integers(0, 2**32, (blocks, words_per_block), dtype=np.uint64).astype(np.uint32)
    return keys, words


# --------------------------------------------------------------------------
# Workload families (instance batches); parameters per family are the
# search parameters of Table 2 where the paper gives them.
# --------------------------------------------------------------------------
def search_params(n_activities: int) -> tuple:
    """(swap distance, tabu list length) by instance size: the single-instance
    workload's (20, 60) up to 45 activities, then Table 2's rows."""
    if n_activities <= 45:
        return 20, 60
    if n_activities <= 75:
        return 60, 250
    if n_activities <= 105:
        return 60, 600
    return 60, 800


def config_batch(name: str, count: Optional[int] = None, first: int = 0) -> List[Instance]:
    """Instances of a named workload.

    ``j30_single``  -- seed 0, n=30, M=4, NC=1.5, RS=0.5
    ``j30_batch``   -- seeds 0.., n=30, M=4, NC over NC_GRID, RS over RS_GRID4
    ``j120_batch``  -- seeds 0.., n=120, M=4, NC over NC_GRID, RS over RS_GRID5
    ``mixed_batch`` -- n from {30,60,90,120,300}, M in [4,8], d in [1,50]
    """
    out = []
    if name == "j30_single":
        return [generate(0, 30, 4, 150, 50, stream=1)]
    if name == "j30_batch":
        count = 480 if count is None else count
        for s in range(first, first + count):
            out.append(generate(s, 30, 4, NC_GRID[s % 3], RS_GRID4[(s // 3) % 4], stream=2))
        return out
    if name == "j120_batch":
        count = 600 if count is None else count
        for s in range(first, first + count):
            out.append(generate(s, 120, 4, NC_GRID[s % 3], RS_GRID5[(s // 3) % 5], stream=3))
        return out
    if name == "mixed_batch":
        count = 1024 if count is None else count
        for s in range(first, first + count):
            rng = np.random.Generator(np.random.Philox(key=[s, 4]))
            n = int(rng.choice([30, 60, 90, 120, 300]))
            m = int(rng.integers(4, 9))
            out.append(generate(s, n, m, NC_GRID[s % 3], RS_GRID4[(s // 3) % 4],
                                dmin=1, dmax=50, stream=4))
        return out
    raise ValueError(f"unknown workload {name!r}")
