"""CPU tests of the C library's host logic and interface (no GPU calls).

The library must load and export every function include/rcpsp.h declares;
the host preparation (validation, critical path, initial list, evaluator
choice) runs without a GPU through rcpsp_prepare_instance and is compared
with the CPU reference; invalid instances must be rejected with the
documented codes.
"""
import os
import re

import numpy as np
import pytest

from paper_1711_04556_gb300 import build as B
from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return R.library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rcpsp.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(rcpsp_\w+)\(", text, re.M)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(R.EXPORTS) == names


def test_prepare_matches_oracle(lib, oracle):
    insts = (I.config_batch("j30_batch", 24) + I.config_batch("j120_batch", 6)
             + I.config_batch("mixed_batch", 6)
             + [I.generate(s, 12, 3, 180, 50, relabel=True, stream=7) for s in range(10)])
    for k, inst in enumerate(insts):
        key = I.level_keys(inst, k) if k % 2 else None
        p = R.prepare(inst, key)
        assert p["cp"] == oracle.critical_path(inst)
        assert p["ub"] == int(inst.dur.sum())
        assert p["initial"].tolist() == oracle.initial_order(inst, key).tolist()
        assert p["mode"] == oracle.select_mode(inst)


def test_table1_prepare(lib):
    p = R.prepare(I.table1_instance())
    assert p["cp"] == 16 and p["ub"] == 35 and p["mode"] == R.EVAL_TIME


def _mutate(inst, **kw):
    d = dict(n=inst.n, m=inst.m, dur=inst.dur.copy(), cap=inst.cap.copy(), req=inst.req.copy(),
             succ_off=inst.succ_off.copy(), succ=inst.succ.copy())
    d.update(kw)
    return I.Instance(**d)


def _code(inst):
    with pytest.raises(R.RcpspError) as e:
        R.prepare(inst)
    return e.value.code


def test_validation_codes(lib):
    base = I.generate(1, 8, 2, 150, 50, stream=5)
    n, m = base.n, base.m
    # cycle: add arc from the last non-dummy activity back to activity 1
    succ_sets = [list(base.successors(i)) for i in range(n)]
    src = next(i for i in range(1, n - 1) if (n - 1) in succ_sets[i])
    succ_sets[src].append(1) if 1 not in succ_sets[src] and src != 1 else None
    if src != 1:
        off = np.r_[0, np.cumsum([len(s) for s in succ_sets])].astype(np.int32)
        cyc = _mutate(base, succ_off=off, succ=np.array([x for s in succ_sets for x in s], np.int32))
        assert _code(cyc) in (-2, -3)
    dur = base.dur.copy(); dur[0] = 1
    assert _code(_mutate(base, dur=dur)) == -3
    req = base.req.copy(); req[m] = base.cap[0] + 1
    assert _code(_mutate(base, req=req)) == -4
    req = base.req.copy(); req[(n - 1) * m] = 1
    assert _code(_mutate(base, req=req)) in (-3, -4)
    dur = base.dur.copy(); dur[1] = -1
    assert _code(_mutate(base, dur=dur)) == -1
    dur = base.dur.copy(); dur[1] = 40000
    assert _code(_mutate(base, dur=dur)) == -5
    cap = base.cap.copy(); cap[0] = 0
    assert _code(_mutate(base, cap=cap)) == -1
    succ = base.succ.copy(); succ[0] = n + 5
    assert _code(_mutate(base, succ=succ)) == -1
    big = I.generate(0, 3, 9, 150, 50, stream=5)
    assert _code(big) == -5                                  # M > 8
    tiny = I.Instance(2, 1, np.zeros(2, np.int32), np.ones(1, np.int32), np.zeros(2, np.int32),
                      np.array([0, 1, 1], np.int32), np.array([1], np.int32))
    assert _code(tiny) == -1                                 # N < 3
    # an activity without a successor (not connected to the sink)
    succ_sets = [list(base.successors(i)) for i in range(n)]
    j = next(i for i in range(1, n - 1) if succ_sets[i] == [n - 1])
    succ_sets[j] = []
    off = np.r_[0, np.cumsum([len(s) for s in succ_sets])].astype(np.int32)
    assert _code(_mutate(base, succ_off=off, succ=np.array([x for s in succ_sets for x in s], np.int32))) == -3


def test_generator_is_deterministic():
    a = I.config_batch("j30_batch", 5)
    b = I.config_batch("j30_batch", 5)
    assert [x.digest() for x in a] == [x.digest() for x in b]
    assert len({x.digest() for x in a}) == 5
    x = I.generate(3, 30, 4, 210, 20)
    assert x.n == 32 and x.dur[0] == 0 and x.dur[-1] == 0
    assert int(np.sum(x.succ_off[1:-1] - x.succ_off[:-2] > 0)) >= 30   # every non-dummy has a successor
    t = I.Instance.from_text(x.to_text())
    assert t.digest() == x.digest()


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes mirror of a public struct has the C size and the C
    offset of each field (a C program compiled against include/rcpsp.h
    prints them)."""
    import ctypes as C
    import subprocess
    from paper_1711_04556_gb300 import rcpsp as R
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    mirrors = {"rcpsp_instance": R.Instance, "rcpsp_params": R.Params, "rcpsp_coop_params": R.CoopParams,
               "rcpsp_stats": R.Stats, "rcpsp_allocator": R.Allocator, "rcpsp_server_config": R.ServerConfig,
               "rcpsp_completion": R.Completion, "rcpsp_server_stats": R.ServerStats, "rcpsp_peaks": R.Peaks,
               "rcpsp_launch_info": R.LaunchInfo}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rcpsp.h"', 'int main(void) {']
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
    # the numpy images used to fill and read many records at once
    for dt, cname in ((R._INSTANCE_DTYPE, "rcpsp_instance"), (R._STATS_DTYPE, "rcpsp_stats")):
        assert dt.itemsize == got[(cname, "sizeof")]
        for field in dt.names:
            assert dt.fields[field][1] == got[(cname, field)], (cname, field)


def _reaches_avoiding(succ, a, b):
    """b reachable from a by a path of two or more arcs."""
    stack = [x for x in succ[a] if x != b]
    seen = set(stack)
    while stack:
        x = stack.pop()
        if x == b:
            return True
        for y in succ[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return False


def test_generator_follows_the_stated_recipe():
    """Durations and demands in range (demands used with probability 0.5),
    round(NC n) arcs among the non-dummy activities, a transitively reduced
    graph with the source and sink joined to exactly the activities without
    predecessors / successors, the capacities of the resource-strength
    formula from the earliest-start profile, and the parameter grid of the
    batches."""
    from fractions import Fraction
    used = cells = 0
    fams = (("j30_batch", 48, 10), ("j120_batch", 10, 10), ("mixed_batch", 12, 50))
    for fam, cnt, dmax in fams:
        for s, x in enumerate(I.config_batch(fam, cnt)):
            N, m, n = x.n, x.m, x.n - 2
            nc, rs = x.meta["nc100"], x.meta["rs100"]
            if fam == "j30_batch":
                assert (nc, rs) == ((150, 180, 210)[s % 3], (20, 50, 70, 100)[(s // 3) % 4])
            assert x.dur[0] == 0 and x.dur[-1] == 0 and 1 <= x.dur[1:-1].min() and x.dur.max() <= dmax
            req = x.req.reshape(N, m)
            assert not req[0].any() and not req[-1].any()
            assert ((req[1:-1] == 0) | ((req[1:-1] >= 1) & (req[1:-1] <= 10))).all()
            used += int((req[1:-1] > 0).sum())
            cells += n * m
            succ = [list(x.successors(i)) for i in range(N)]
            pred = [[] for _ in range(N)]
            for a, b in x.arcs():
                pred[b].append(a)
            inner = [(a, b) for a, b in x.arcs() if a != 0 and b != N - 1]
            assert len(inner) == (nc * n + 50) // 100
            for i in range(1, N - 1):
                assert (0 in pred[i]) == (not [p for p in pred[i] if p != 0])
                assert (N - 1 in succ[i]) == (not [q for q in succ[i] if q != N - 1])
            for a, b in x.arcs():
                assert not _reaches_avoiding(succ, a, b), (fam, s, a, b)
            # earliest starts in a topological order of the arcs (Kahn)
            indeg = [len(p) for p in pred]
            order, ready = [], [0]
            while ready:
                a = ready.pop()
                order.append(a)
                for b in succ[a]:
                    indeg[b] -= 1
                    if indeg[b] == 0:
                        ready.append(b)
            assert len(order) == N
            es = [0] * N
            for a in order:
                for b in succ[a]:
                    es[b] = max(es[b], es[a] + int(x.dur[a]))
            for k in range(m):
                kmin = int(req[:, k].max())
                if kmin == 0:
                    assert x.cap[k] == 1
                    continue
                kmax = max(sum(int(req[i, k]) for i in range(N) if es[i] <= t < es[i] + x.dur[i])
                           for t in range(max(es) + 1))
                want = kmin + int(Fraction(rs, 100) * (kmax - kmin) + Fraction(1, 2))
                assert x.cap[k] == want, (fam, s, k)
    assert abs(used / cells - 0.5) < 0.03
