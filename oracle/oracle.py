"""ctypes front end of the CPU reference (oracle) library.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg.  The product path never imports this module.

The C sources sit beside this file; ``build()`` compiles them with the host
compiler (plain C, -O2, no target-specific flags, no floating-point
contraction) into
``librcpsp_oracle.so`` next to them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rcpsp_oracle.c")
HDR = os.path.join(HERE, "rcpsp_oracle.h")
LIB = os.path.join(HERE, "librcpsp_oracle.so")

AUTO, TIME, CAPACITY = 0, 1, 2
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its sources."""
    with _lock:
        stale = (not os.path.exists(LIB) or force or
                 os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
        if stale:
            tmp = LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
                            "-Wall", "-Wextra", "-o", tmp, SRC], check=True)
            os.replace(tmp, LIB)
    return LIB


class _Inst(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int),
                ("dur", C.POINTER(C.c_int)), ("cap", C.POINTER(C.c_int)),
                ("req", C.POINTER(C.c_int)), ("succ_off", C.POINTER(C.c_int)),
                ("succ", C.POINTER(C.c_int)), ("level_key", C.POINTER(C.c_int))]


class _Params(C.Structure):
    _fields_ = [("iterations", C.c_int), ("max_swap_dist", C.c_int), ("tabu_len", C.c_int),
                ("eval_mode", C.c_int), ("stop_at_cp", C.c_int)]


class _CoopParams(C.Structure):
    _fields_ = [("blocks", C.c_int), ("working_set", C.c_int), ("phi_max", C.c_int),
                ("phi_steps", C.c_int), ("assign_fixed", C.c_int), ("words_per_block", C.c_int),
                ("fbi_every", C.c_int)]


class _CoopEvent(C.Structure):
    _fields_ = [("iteration", C.c_int), ("block", C.c_int), ("kind", C.c_int), ("slot", C.c_int),
                ("cmax", C.c_int), ("assigned", C.c_int), ("diversified", C.c_int), ("phi", C.c_int),
                ("ic", C.c_longlong)]


class _Result(C.Structure):
    _fields_ = [("best_W", C.POINTER(C.c_int)), ("best_S", C.POINTER(C.c_int)),
                ("trace", C.POINTER(C.c_int)), ("best_cmax", C.c_int),
                ("iterations", C.c_int), ("mode", C.c_int), ("cp", C.c_int),
                ("evaluated", C.c_longlong), ("work", C.c_longlong), ("status", C.c_int)]


def load(path: str):
    """Opens an oracle library at ``path`` and declares its signatures."""
    h = C.CDLL(path)
    P = C.POINTER
    sig = {
        "orc_check_schedule": (C.c_int, [P(_Inst), P(C.c_int), P(C.c_int)]),
        "orc_critical_path": (C.c_int, [P(_Inst)]),
        "orc_levels": (C.c_int, [P(_Inst), P(C.c_int)]),
        "orc_initial_order": (C.c_int, [P(_Inst), P(C.c_int)]),
        "orc_move_feasible": (C.c_int, [P(_Inst), P(C.c_int), C.c_int, C.c_int]),
        "orc_decode_time": (C.c_int, [P(_Inst), P(C.c_int), P(C.c_int), P(C.c_longlong)]),
        "orc_decode_capacity": (C.c_int, [P(_Inst), P(C.c_int), P(C.c_int), P(C.c_longlong)]),
        "orc_capacity_update": (C.c_int, [P(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int]),
        "orc_select_mode": (C.c_int, [P(_Inst)]),
        "orc_tabu_search": (C.c_int, [P(_Inst), P(_Params), P(_Result)]),
        "orc_tabu_search_batch": (C.c_int, [P(_Inst), C.c_int, P(_Params), P(_Result), C.c_int]),
        "orc_fbi": (C.c_int, [P(_Inst), C.c_int, P(C.c_int), P(C.c_int)]),
        "orc_fbi_pass": (C.c_int, [P(_Inst), C.c_int, P(C.c_int), P(C.c_int), P(C.c_int), P(C.c_int)]),
        "orc_exp_neg": (C.c_double, [C.c_double]),
        "orc_assigned_iterations": (C.c_int, [C.c_int, C.c_int, C.c_longlong, C.c_int]),
        "orc_diversify": (C.c_int, [P(_Inst), P(C.c_int), C.c_int, C.c_int, P(C.c_uint), C.c_int,
                                    P(C.c_int)]),
        "orc_coop_search": (C.c_int, [P(_Inst), P(_Params), P(_CoopParams), P(P(C.c_int)), P(C.c_uint),
                                      P(_Result), P(_CoopEvent), C.c_int, P(C.c_int)]),
        "orc_brute_force_lists": (C.c_int, [P(_Inst), C.c_int, P(C.c_longlong)]),
        "orc_brute_force_starts": (C.c_int, [P(_Inst)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(h, name)
        f.restype, f.argtypes = res, args
    return h


def _lib():
    global _handle
    if _handle is None:
        build()
        _handle = load(LIB)
    return _handle


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class _Marshalled:
    """Keeps the int32 copies alive for as long as the C struct is used."""

    def __init__(self, inst, level_key=None):
        self.arrs = [np.ascontiguousarray(x, np.int32) for x in
                     (inst.dur, inst.cap, inst.req, inst.succ_off, inst.succ)]
        self.key = None if level_key is None else np.ascontiguousarray(level_key, np.int32)
        self.s = _Inst(inst.n, inst.m, *[_ip(a) for a in self.arrs],
                       _ip(self.key) if self.key is not None else None)


def check_schedule(inst, S) -> tuple:
    mi = _Marshalled(inst)
    S = np.ascontiguousarray(S, np.int32)
    cm = C.c_int(0)
    rc = _lib().orc_check_schedule(C.byref(mi.s), _ip(S), C.byref(cm))
    return rc, cm.value


def critical_path(inst) -> int:
    return _lib().orc_critical_path(C.byref(_Marshalled(inst).s))


def levels(inst) -> np.ndarray:
    out = np.zeros(inst.n, np.int32)
    if _lib().orc_levels(C.byref(_Marshalled(inst).s), _ip(out)) != 0:
        raise ValueError("cycle")
    return out


def initial_order(inst, level_key=None) -> np.ndarray:
    out = np.zeros(inst.n, np.int32)
    if _lib().orc_initial_order(C.byref(_Marshalled(inst, level_key).s), _ip(out)) != 0:
        raise ValueError("cycle")
    return out


def move_feasible(inst, W, u, v) -> bool:
    W = np.ascontiguousarray(W, np.int32)
    return bool(_lib().orc_move_feasible(C.byref(_Marshalled(inst).s), _ip(W), u, v))


def decode(inst, W, mode: int) -> tuple:
    """Returns (C_max, S, work) with the chosen decoder (TIME or CAPACITY)."""
    W = np.ascontiguousarray(W, np.int32)
    S = np.zeros(inst.n, np.int32)
    work = C.c_longlong(0)
    f = _lib().orc_decode_time if mode == TIME else _lib().orc_decode_capacity
    c = f(C.byref(_Marshalled(inst).s), _ip(W), _ip(S), C.byref(work))
    return c, S, work.value


def capacity_update(c, R: int, r: int, d: int, s: int) -> tuple:
    arr = np.ascontiguousarray(c, np.int32).copy()
    steps = _lib().orc_capacity_update(_ip(arr), R, r, d, s)
    return arr, steps


def select_mode(inst) -> int:
    return _lib().orc_select_mode(C.byref(_Marshalled(inst).s))


def _result_buffers(n, iterations, trace):
    W = np.zeros(n, np.int32)
    S = np.zeros(n, np.int32)
    T = np.zeros(max(1, 3 * iterations), np.int32) if trace else None
    r = _Result(_ip(W), _ip(S), _ip(T) if T is not None else None, 0, 0, 0, 0, 0, 0, 0)
    return r, W, S, T


def _to_dict(r, W, S, T):
    d = dict(best_W=W, best_S=S, best_cmax=r.best_cmax, iterations=r.iterations, mode=r.mode,
             cp=r.cp, evaluated=r.evaluated, work=r.work, status=r.status)
    if T is not None:
        d["trace"] = T[:3 * r.iterations].reshape(-1, 3)
    return d


def tabu_search(inst, iterations=100, delta=20, tabu_len=60, mode=AUTO, stop_at_cp=1,
                trace=False, level_key=None) -> dict:
    mi = _Marshalled(inst, level_key)
    p = _Params(iterations, delta, tabu_len, mode, stop_at_cp)
    r, W, S, T = _result_buffers(inst.n, iterations, trace)
    _lib().orc_tabu_search(C.byref(mi.s), C.byref(p), C.byref(r))
    return _to_dict(r, W, S, T)


def tabu_search_batch(insts: Sequence, params: Sequence[tuple], nthreads: int,
                      level_keys: Optional[Sequence] = None, trace=False) -> List[dict]:
    """Independent searches over a host thread pool.

    ``params[k]`` = (iterations, delta, tabu_len, mode, stop_at_cp).  The
    C library takes one parameter set per call, so instances are grouped by
    parameter set.
    """
    out: List[Optional[dict]] = [None] * len(insts)
    groups = {}
    for k, p in enumerate(params):
        groups.setdefault(tuple(p), []).append(k)
    for p, idx in groups.items():
        ms = [_Marshalled(insts[k], None if level_keys is None else level_keys[k]) for k in idx]
        arr = (_Inst * len(idx))(*[m.s for m in ms])
        bufs = [_result_buffers(insts[k].n, p[0], trace) for k in idx]
        res = (_Result * len(idx))(*[b[0] for b in bufs])
        _lib().orc_tabu_search_batch(arr, len(idx), C.byref(_Params(*p)), res, nthreads)
        for j, k in enumerate(idx):
            out[k] = _to_dict(res[j], *bufs[j][1:])
    return out  # type: ignore[return-value]


def brute_force_lists(inst, mode=TIME) -> tuple:
    lists = C.c_longlong(0)
    best = _lib().orc_brute_force_lists(C.byref(_Marshalled(inst).s), mode, C.byref(lists))
    return best, lists.value


def brute_force_starts(inst) -> int:
    return _lib().orc_brute_force_starts(C.byref(_Marshalled(inst).s))


# ---------------------------------------------------------------------------
# Sec. 6.1: co-operating searches (readings C1-C8 in the C source)
# ---------------------------------------------------------------------------
COOP_EVENT_FIELDS = [f for f, _ in _CoopEvent._fields_]


def fbi(inst, W, mode: int) -> tuple:
    """Forward-backward improvement of W; returns (list, C_max, passes)."""
    W = np.array(W, np.int32)
    passes = C.c_int(0)
    c = _lib().orc_fbi(C.byref(_Marshalled(inst).s), mode, _ip(W), C.byref(passes))
    return W, c, passes.value


def fbi_pass(inst, W, mode: int) -> tuple:
    """One FBI pass: (forward list, its C_max, backward makespan T, mirrored backward starts)."""
    W = np.ascontiguousarray(W, np.int32)
    Wn = np.zeros(inst.n, np.int32)
    Sb = np.zeros(inst.n, np.int32)
    T = C.c_int(0)
    c = _lib().orc_fbi_pass(C.byref(_Marshalled(inst).s), mode, _ip(W), _ip(Wn), C.byref(T), _ip(Sb))
    return Wn, c, T.value, Sb


def exp_neg(x: float) -> float:
    return _lib().orc_exp_neg(float(x))


def assigned_iterations(c_k: int, c_star: int, ic_k: int, i_block: int) -> int:
    return _lib().orc_assigned_iterations(int(c_k), int(c_star), int(ic_k), int(i_block))


def diversify(inst, W, delta: int, steps: int, words, cursor: int = 0) -> tuple:
    """Returns (new list, swaps applied, new cursor)."""
    W = np.array(W, np.int32)
    words = np.ascontiguousarray(words, np.uint32)
    cur = C.c_int(cursor)
    done = _lib().orc_diversify(C.byref(_Marshalled(inst).s), _ip(W), delta, steps,
                                words.ctypes.data_as(C.POINTER(C.c_uint)), len(words), C.byref(cur))
    return W, done, cur.value


def coop_search(inst, iterations=100, delta=20, tabu_len=60, mode=AUTO, stop_at_cp=1, blocks=4,
                working_set=16, phi_max=3, phi_steps=20, assign_fixed=0, slot_keys=None, words=None,
                log_cap=0, fbi_every=2) -> dict:
    """B co-operating searches of one instance through a working set of
    `working_set` slots.  slot_keys: None or a list of |F| entries (None or
    N keys).  words: uint32 [blocks, P] random words (None if phi_steps == 0).
    With log_cap > 0 the result carries the exchange events under "log"."""
    mi = _Marshalled(inst)
    p = _Params(iterations, delta, tabu_len, mode, stop_at_cp)
    keep = []
    keys_arr = None
    if slot_keys is not None:
        keys_arr = (C.POINTER(C.c_int) * working_set)()
        for k in range(working_set):
            if slot_keys[k] is not None:
                a = np.ascontiguousarray(slot_keys[k], np.int32)
                keep.append(a)
                keys_arr[k] = _ip(a)
    P = 0
    wptr = None
    if words is not None:
        w = np.ascontiguousarray(words, np.uint32).reshape(blocks, -1)
        keep.append(w)
        P = w.shape[1]
        wptr = w.ctypes.data_as(C.POINTER(C.c_uint))
    cp = _CoopParams(blocks, working_set, phi_max, phi_steps, assign_fixed, P, fbi_every)
    r, W, S, _ = _result_buffers(inst.n, iterations, False)
    ev = (_CoopEvent * max(1, log_cap))()
    n_ev = C.c_int(0)
    _lib().orc_coop_search(C.byref(mi.s), C.byref(p), C.byref(cp), keys_arr, wptr, C.byref(r),
                           ev if log_cap > 0 else None, log_cap, C.byref(n_ev))
    d = _to_dict(r, W, S, None)
    if log_cap > 0:
        d["log"] = [{f: getattr(ev[k], f) for f in COOP_EVENT_FIELDS} for k in range(min(n_ev.value, log_cap))]
        d["log_events"] = n_ev.value
    return d


def coop_search_batch(insts: Sequence, kwargs: Sequence[dict], nthreads: int) -> List[dict]:
    """coop_search over a pool of host threads (the C calls run without the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    _lib()
    with ThreadPoolExecutor(max_workers=max(1, nthreads)) as ex:
        return list(ex.map(lambda a: coop_search(a[0], **a[1]), zip(insts, kwargs)))
