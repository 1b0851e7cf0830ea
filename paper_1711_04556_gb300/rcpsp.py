"""Python binding of the C interface in include/rcpsp.h (argument marshalling only).

Every step of the search runs in the CUDA library; this module converts
numpy arrays to the C structs, hands PyTorch's CUDA caching allocator and
streams to the library, and converts results back.  There is no CPU path:
without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librcpsp_gb300.so")

EVAL_AUTO, EVAL_TIME, EVAL_CAPACITY = 0, 1, 2
E_INVALID_ARG, E_TOO_LARGE, E_NOT_FOUND = -1, -5, -8
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "CYCLE", -3: "DUMMY", -4: "DEMAND_EXCEEDS_CAP",
          -5: "TOO_LARGE", -6: "CUDA", -7: "TIMEOUT", -8: "NOT_FOUND", -9: "DEVICE"}
EXPORTS = ("rcpsp_create", "rcpsp_destroy", "rcpsp_load_instances", "rcpsp_free_instances",
           "rcpsp_tabu_search", "rcpsp_tabu_search_noalloc", "rcpsp_coop_search", "rcpsp_autotune",
           "rcpsp_get_schedules", "rcpsp_get_trace", "rcpsp_evaluate_lists",
           "rcpsp_prepare_instance", "rcpsp_transfer_bytes", "rcpsp_kernel_launches", "rcpsp_get_state",
           "rcpsp_set_state", "rcpsp_measure_peaks", "rcpsp_last_launches", "rcpsp_multistart",
           "rcpsp_server_create", "rcpsp_server_destroy",
           "rcpsp_server_submit", "rcpsp_server_poll", "rcpsp_server_get_stats", "rcpsp_last_error")


class RcpspError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Instance(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("dur", C.POINTER(C.c_int32)),
                ("cap", C.POINTER(C.c_int32)), ("req", C.POINTER(C.c_int32)),
                ("succ_off", C.POINTER(C.c_int32)), ("succ", C.POINTER(C.c_int32)),
                ("level_key", C.POINTER(C.c_int32))]


class Params(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("max_swap_dist", C.c_int32), ("tabu_len", C.c_int32),
                ("eval_mode", C.c_int32), ("stop_at_cp", C.c_int32), ("group_size", C.c_int32),
                ("warps_per_cta", C.c_int32), ("record_trace", C.c_int32), ("use_graph", C.c_int32),
                ("cluster_size", C.c_int32), ("checkpoint", C.c_int32), ("resume", C.c_int32),
                ("slices", C.c_int32)]


class CoopParams(C.Structure):
    _fields_ = [("blocks", C.c_int32), ("working_set", C.c_int32), ("phi_max", C.c_int32),
                ("phi_steps", C.c_int32), ("assign_fixed", C.c_int32), ("words_per_block", C.c_int32),
                ("fbi_every", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("evaluated", C.c_int64), ("work", C.c_int64), ("iterations", C.c_int32),
                ("eval_mode", C.c_int32), ("critical_path", C.c_int32), ("status", C.c_int32),
                ("t_start_ns", C.c_int64), ("t_end_ns", C.c_int64), ("placements", C.c_int64),
                ("steps_done", C.c_int64), ("update_units", C.c_int64), ("succ_pushes", C.c_int64),
                ("kept_words", C.c_int64)]


# numpy image of rcpsp_stats, for reading many at once
_STATS_DTYPE = np.dtype([("evaluated", "<i8"), ("work", "<i8"), ("iterations", "<i4"), ("eval_mode", "<i4"),
                         ("critical_path", "<i4"), ("status", "<i4"), ("t_start_ns", "<i8"), ("t_end_ns", "<i8"),
                         ("placements", "<i8"), ("steps_done", "<i8"), ("update_units", "<i8"),
                         ("succ_pushes", "<i8"), ("kept_words", "<i8")])
assert _STATS_DTYPE.itemsize == C.sizeof(Stats)


class LaunchInfo(C.Structure):
    _fields_ = [("searches", C.c_int32), ("group_size", C.c_int32), ("warps", C.c_int32),
                ("cluster_size", C.c_int32), ("ctas", C.c_int32), ("prefix_reuse", C.c_int32),
                ("shape_source", C.c_int32), ("slices", C.c_int32), ("smem_bytes", C.c_int64)]


class Peaks(C.Structure):
    _fields_ = [("int32_ops_per_s", C.c_double), ("smem_bytes_per_s", C.c_double), ("int32_ms", C.c_double),
                ("smem_ms", C.c_double), ("sms", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("memory_budget", C.c_int64),
                ("poll_us", C.c_int32), ("slice_iterations", C.c_int32), ("max_pending", C.c_int32)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_int64), ("n", C.c_int32), ("status", C.c_int32), ("best_cmax", C.c_int32),
                ("iterations", C.c_int32), ("eval_mode", C.c_int32), ("critical_path", C.c_int32),
                ("evaluated", C.c_int64), ("work", C.c_int64), ("t_submit_ns", C.c_int64),
                ("t_launch_ns", C.c_int64), ("t_done_ns", C.c_int64), ("order", C.POINTER(C.c_int32)),
                ("start", C.POINTER(C.c_int32))]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "rejected", "admitted", "completed", "batches",
                                         "inflight_requests", "pending", "inflight_bytes",
                                         "max_inflight_bytes", "evaluated", "requeued")]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", FREE_FN), ("user", C.c_void_p)]


_lib_handle = None


def library(path: Optional[str] = None):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib_handle
    if _lib_handle is not None and path is None:
        return _lib_handle
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: build it with paper_1711_04556_gb300.build.build()")
    h = C.CDLL(p)
    P = C.POINTER
    sig = {
        "rcpsp_create": (C.c_int, [P(C.c_void_p), C.c_int, P(Allocator)]),
        "rcpsp_destroy": (C.c_int, [C.c_void_p]),
        "rcpsp_load_instances": (C.c_int, [C.c_void_p, P(Instance), C.c_int32, P(C.c_int32)]),
        "rcpsp_free_instances": (C.c_int, [C.c_void_p, P(C.c_int32), C.c_int32]),
        "rcpsp_tabu_search": (C.c_int, [C.c_void_p, P(C.c_int32), C.c_int32, P(Params), C.c_void_p]),
        "rcpsp_tabu_search_noalloc": (C.c_int, [C.c_void_p, P(C.c_int32), C.c_int32, P(Params), C.c_void_p]),
        "rcpsp_coop_search": (C.c_int, [C.c_void_p, P(C.c_int32), C.c_int32, P(Params), P(CoopParams),
                                        P(C.c_int32), P(C.c_uint32), C.c_void_p]),
        "rcpsp_autotune": (C.c_int, [C.c_void_p, P(C.c_int32), C.c_int32, P(Params), C.c_int32, C.c_void_p,
                                     P(C.c_int32), P(C.c_int32), P(C.c_int32)]),
        "rcpsp_get_schedules": (C.c_int, [C.c_void_p, P(C.c_int32), C.c_int32, P(C.c_int32), P(C.c_int32),
                                          P(C.c_int32), P(Stats)]),
        "rcpsp_get_trace": (C.c_int, [C.c_void_p, C.c_int32, P(C.c_int32), C.c_int32, P(C.c_int32)]),
        "rcpsp_evaluate_lists": (C.c_int, [C.c_void_p, C.c_int32, P(C.c_int32), C.c_int32, C.c_int32,
                                           P(C.c_int32), P(C.c_int32), P(C.c_int64), C.c_void_p]),
        "rcpsp_prepare_instance": (C.c_int, [P(Instance), P(C.c_int32), P(C.c_int32), P(C.c_int32),
                                             P(C.c_int32), C.c_char_p, C.c_int32]),
        "rcpsp_transfer_bytes": (C.c_int, [C.c_void_p, P(C.c_int64), P(C.c_int64)]),
        "rcpsp_kernel_launches": (C.c_int, [C.c_void_p, P(C.c_int64)]),
        "rcpsp_measure_peaks": (C.c_int, [C.c_int, P(Peaks)]),
        "rcpsp_last_launches": (C.c_int, [C.c_void_p, P(LaunchInfo), C.c_int32, P(C.c_int32)]),
        "rcpsp_multistart": (C.c_int, [C.c_void_p, P(Instance), C.c_int32, P(C.c_int32), P(Params), C.c_void_p,
                                       P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_int32), P(Stats)]),
        "rcpsp_get_state": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, P(C.c_size_t)]),
        "rcpsp_set_state": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t]),
        "rcpsp_server_create": (C.c_int, [P(C.c_void_p), C.c_int, P(ServerConfig)]),
        "rcpsp_server_destroy": (C.c_int, [C.c_void_p]),
        "rcpsp_server_submit": (C.c_int, [C.c_void_p, P(Instance), P(Params), C.c_int64]),
        "rcpsp_server_poll": (C.c_int, [C.c_void_p, P(Completion), C.c_int32, P(C.c_int32), C.c_int32]),
        "rcpsp_server_get_stats": (C.c_int, [C.c_void_p, P(ServerStats)]),
        "rcpsp_last_error": (C.c_char_p, [C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(h, name)
        f.restype, f.argtypes = res, args
    if path is None:
        _lib_handle = h
    return h


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: np.ndarray, ty=C.c_int32):
    return a.ctypes.data_as(C.POINTER(ty))


class _Marshalled:
    def __init__(self, inst, level_key=None):
        self.arrs = [_i32(x) for x in (inst.dur, inst.cap, inst.req, inst.succ_off, inst.succ)]
        self.key = None if level_key is None else _i32(level_key)
        self.s = Instance(inst.n, inst.m, *[_ptr(a) for a in self.arrs],
                          _ptr(self.key) if self.key is not None else None)


# numpy image of rcpsp_instance: two int32 then six pointers
_INSTANCE_DTYPE = np.dtype([("n", "<i4"), ("m", "<i4"), ("dur", "<u8"), ("cap", "<u8"), ("req", "<u8"),
                            ("succ_off", "<u8"), ("succ", "<u8"), ("level_key", "<u8")])
assert _INSTANCE_DTYPE.itemsize == C.sizeof(Instance)


class _BatchMarshalled:
    """rcpsp_instance array for many instances: each field is concatenated
    once and the structs are filled with vectorized pointer arithmetic."""

    def __init__(self, instances, level_keys=None):
        cnt = len(instances)
        self.keep = []
        self.rec = np.zeros(cnt, _INSTANCE_DTYPE)
        self.rec["n"] = [x.n for x in instances]
        self.rec["m"] = [x.m for x in instances]
        for field in ("dur", "cap", "req", "succ_off", "succ"):
            parts = [getattr(x, field) for x in instances]
            flat = np.ascontiguousarray(np.concatenate(parts), dtype=np.int32)
            lens = np.fromiter((len(a) for a in parts), np.int64, cnt)
            offs = np.concatenate(([0], np.cumsum(lens)[:-1])) if cnt else np.zeros(0, np.int64)
            self.rec[field] = flat.ctypes.data + 4 * offs
            self.keep.append(flat)
        if level_keys is not None:
            for k, key in enumerate(level_keys):
                if key is not None:
                    a = _i32(key)
                    self.keep.append(a)
                    self.rec["level_key"][k] = a.ctypes.data
        self.ptr = self.rec.ctypes.data_as(C.POINTER(Instance))


def _torch_allocator():
    """Device memory from PyTorch's caching allocator."""
    import torch

    live = {}

    def alloc(nbytes, stream, user):
        try:
            dev = torch.cuda.current_device()
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
            live[p] = nbytes
            return p
        except Exception:  # the library reports the failure as RCPSP_E_CUDA
            return None

    def release(ptr, nbytes, stream, user):
        if ptr in live:
            del live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(release)


def measure_peaks(device: int = 0, lib_path: Optional[str] = None) -> dict:
    """rcpsp_measure_peaks: the measured integer-ALU and shared-memory ceilings."""
    lib = library(lib_path)
    pk = Peaks()
    rc = lib.rcpsp_measure_peaks(device, C.byref(pk))
    if rc != 0:
        raise RcpspError(rc, "rcpsp_measure_peaks failed")
    return {f: getattr(pk, f) for f, _ in Peaks._fields_}


def prepare(inst, level_key=None, lib_path: Optional[str] = None) -> dict:
    """Host preparation of one instance without a GPU (rcpsp_prepare_instance)."""
    lib = library(lib_path)
    m = _Marshalled(inst, level_key)
    cp, ub, mode = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    W = np.zeros(inst.n, np.int32)
    msg = C.create_string_buffer(256)
    rc = lib.rcpsp_prepare_instance(C.byref(m.s), C.byref(cp), C.byref(ub), _ptr(W), C.byref(mode), msg, 256)
    if rc != 0:
        raise RcpspError(rc, msg.value.decode())
    return dict(cp=cp.value, ub=ub.value, initial=W, mode=mode.value)


class Solver:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, torch_memory: bool = True, lib_path: Optional[str] = None):
        self.lib = library(lib_path)
        self.ctx = C.c_void_p()
        self._cbs = None
        alloc = None
        if torch_memory:
            import torch
            torch.cuda.set_device(device)
            self._cbs = _torch_allocator()
            alloc = Allocator(self._cbs[0], self._cbs[1], None)
        self._check(self.lib.rcpsp_create(C.byref(self.ctx), device, C.byref(alloc) if alloc else None))
        self.n_of = {}

    def _check(self, rc: int):
        if rc != 0:
            msg = self.lib.rcpsp_last_error(self.ctx).decode() if self.ctx else ""
            raise RcpspError(rc, msg)

    def close(self):
        if self.ctx:
            self.lib.rcpsp_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ calls
    def load(self, instances: Sequence, level_keys: Optional[Sequence] = None) -> np.ndarray:
        bm = _BatchMarshalled(instances, level_keys)
        ids = np.zeros(len(instances), np.int32)
        self._check(self.lib.rcpsp_load_instances(self.ctx, bm.ptr, len(instances), _ptr(ids)))
        for i, x in zip(ids, instances):
            self.n_of[int(i)] = x.n
        return ids

    def free(self, ids):
        ids = _i32(ids)
        self._check(self.lib.rcpsp_free_instances(self.ctx, _ptr(ids), len(ids)))
        for i in ids:
            self.n_of.pop(int(i), None)

    def search(self, ids, iterations: int = 100, delta: int = 0, tabu_len: int = 0, mode: int = EVAL_AUTO,
               stop_at_cp: bool = True, group_size: int = 0, warps_per_cta: int = 0, trace: bool = False,
               use_graph: bool = False, stream=None, cluster_size: int = 0, checkpoint: bool = False,
               resume: bool = False, slices: int = 0):
        """Asynchronous search on ``stream`` (a torch.cuda.Stream, a raw handle or None).
        checkpoint keeps each search's state on the device; resume continues it;
        slices: 0 automatic, 1 none, k: every search in k slices (same results)."""
        ids = _i32(ids)
        p = Params(iterations, delta, tabu_len, mode, int(stop_at_cp), group_size, warps_per_cta,
                   int(trace), int(use_graph), cluster_size, int(checkpoint), int(resume), slices)
        handle = getattr(stream, "cuda_stream", stream) or None
        self._check(self.lib.rcpsp_tabu_search(self.ctx, _ptr(ids), len(ids), C.byref(p), handle))

    def coop_search(self, ids, iterations: int = 100, delta: int = 0, tabu_len: int = 0, mode: int = EVAL_AUTO,
                    stop_at_cp: bool = True, blocks: int = 4, working_set: int = 16, phi_max: int = 3,
                    phi_steps: int = 20, assign_fixed: int = 0, slot_keys=None, words=None,
                    group_size: int = 0, warps_per_cta: int = 0, stream=None, fbi_every: int = 2):
        """rcpsp_coop_search: `blocks` co-operating searches per instance.

        slot_keys: None, or per instance a list of `working_set` entries
        (None = unshuffled, else N keys).  words: None, or per instance a
        uint32 array [blocks, P] (required when phi_steps > 0)."""
        ids = _i32(ids)
        keys = None
        if slot_keys is not None:
            rows = []
            for i, per in zip(ids, slot_keys):
                n = self.n_of[int(i)]
                for f in range(working_set):
                    k = per[f] if per is not None else None
                    rows.append(np.zeros(n, np.int32) if k is None else np.asarray(k, np.int32))
            keys = np.ascontiguousarray(np.concatenate(rows), np.int32)
        wp, P = None, 0
        if words is not None:
            w = np.ascontiguousarray(np.stack([np.asarray(x, np.uint32).reshape(blocks, -1) for x in words]))
            P = w.shape[2]
            wp = w.ctypes.data_as(C.POINTER(C.c_uint32))
        p = Params(iterations, delta, tabu_len, mode, int(stop_at_cp), group_size, warps_per_cta, 0, 0, 0)
        cp = CoopParams(blocks, working_set, phi_max, phi_steps, assign_fixed, P, fbi_every)
        handle = getattr(stream, "cuda_stream", stream) or None
        self._check(self.lib.rcpsp_coop_search(self.ctx, _ptr(ids), len(ids), C.byref(p), C.byref(cp),
                                               _ptr(keys) if keys is not None else None, wp, handle))

    def search_noalloc(self, ids, iterations: int = 100, delta: int = 0, tabu_len: int = 0,
                       mode: int = EVAL_AUTO, stop_at_cp: bool = True, group_size: int = 0,
                       warps_per_cta: int = 0, stream=None):
        """rcpsp_tabu_search_noalloc: the search without any device allocation."""
        ids = _i32(ids)
        p = Params(iterations, delta, tabu_len, mode, int(stop_at_cp), group_size, warps_per_cta, 0, 0, 1)
        handle = getattr(stream, "cuda_stream", stream) or None
        self._check(self.lib.rcpsp_tabu_search_noalloc(self.ctx, _ptr(ids), len(ids), C.byref(p), handle))

    def autotune(self, ids, iterations: int = 100, delta: int = 0, tabu_len: int = 0, mode: int = EVAL_AUTO,
                 stop_at_cp: bool = True, trial_iterations: int = 48, stream=None):
        """rcpsp_autotune: times trial searches of every launch shape; returns
        (group_size, warps, cluster_size) of the largest launch class."""
        ids = _i32(ids)
        p = Params(iterations, delta, tabu_len, mode, int(stop_at_cp), 0, 0, 0, 0, 0)
        g, w, cs = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        handle = getattr(stream, "cuda_stream", stream) or None
        self._check(self.lib.rcpsp_autotune(self.ctx, _ptr(ids), len(ids), C.byref(p), trial_iterations, handle,
                                            C.byref(g), C.byref(w), C.byref(cs)))
        return g.value, w.value, cs.value

    def results(self, ids) -> List[dict]:
        ids = _i32(ids)
        ns = [self.n_of[int(i)] for i in ids]
        tot = int(sum(ns))
        order = np.zeros(tot, np.int32)
        start = np.zeros(tot, np.int32)
        cmax = np.zeros(len(ids), np.int32)
        st = np.zeros(len(ids), _STATS_DTYPE)
        self._check(self.lib.rcpsp_get_schedules(self.ctx, _ptr(ids), len(ids), _ptr(order), _ptr(start),
                                                 _ptr(cmax), st.ctypes.data_as(C.POINTER(Stats))))
        cols = [st[f].tolist() for f in _STATS_DTYPE.names]
        cm = cmax.tolist()
        out, at = [], 0
        for k, n in enumerate(ns):
            ev, wk, it, md, cp, stt, t0, t1, pl, sd, ud, sp, kw = (c[k] for c in cols)
            out.append(dict(best_W=order[at:at + n], best_S=start[at:at + n], best_cmax=cm[k], evaluated=ev,
                            work=wk, iterations=it, mode=md, cp=cp, status=stt, t_start_ns=t0, t_end_ns=t1,
                            placements=pl, steps_done=sd, update_units=ud, succ_pushes=sp, kept_words=kw))
            at += n
        return out

    def transfer_bytes(self):
        h2d, d2h = C.c_int64(0), C.c_int64(0)
        self._check(self.lib.rcpsp_transfer_bytes(self.ctx, C.byref(h2d), C.byref(d2h)))
        return h2d.value, d2h.value

    def get_state(self, id_: int) -> bytes:
        """rcpsp_get_state: the kept search state of instance `id_`."""
        size = C.c_size_t(0)
        self._check(self.lib.rcpsp_get_state(self.ctx, int(id_), None, 0, C.byref(size)))
        buf = (C.c_char * size.value)()
        self._check(self.lib.rcpsp_get_state(self.ctx, int(id_), buf, size.value, C.byref(size)))
        return bytes(buf)

    def set_state(self, id_: int, state: bytes) -> None:
        """rcpsp_set_state: give instance `id_` a kept state (from get_state)."""
        buf = C.create_string_buffer(state, len(state))
        self._check(self.lib.rcpsp_set_state(self.ctx, int(id_), buf, len(state)))

    def multistart(self, inst, level_keys, iterations: int = 1000, delta: int = 0, tabu_len: int = 0,
                   mode: int = EVAL_AUTO, stop_at_cp: bool = True, stream=None) -> dict:
        """rcpsp_multistart: one search per row of level_keys (None = the
        unshuffled order); the best start's result and every start's makespan."""
        starts = len(level_keys)
        keys = np.zeros((starts, inst.n), np.int32)
        for k, key in enumerate(level_keys):
            if key is not None:
                keys[k] = _i32(key)
        m = _Marshalled(inst)
        p = Params(iterations, delta, tabu_len, mode, int(stop_at_cp), 0, 0, 0, 0, 0)
        best = C.c_int32(0)
        order = np.zeros(inst.n, np.int32)
        start = np.zeros(inst.n, np.int32)
        makespans = np.zeros(starts, np.int32)
        st = np.zeros(1, _STATS_DTYPE)
        handle = getattr(stream, "cuda_stream", stream) or None
        self._check(self.lib.rcpsp_multistart(self.ctx, C.byref(m.s), starts, _ptr(keys), C.byref(p), handle,
                                              C.byref(best), _ptr(order), _ptr(start), _ptr(makespans),
                                              st.ctypes.data_as(C.POINTER(Stats))))
        out = {f: st[f][0].item() for f in _STATS_DTYPE.names}
        return dict(start=best.value, best_W=order, best_S=start, best_cmax=int(makespans[best.value]),
                    makespans=makespans.tolist(), evaluated=out["evaluated"], work=out["work"],
                    iterations=out["iterations"], mode=out["eval_mode"], cp=out["critical_path"],
                    status=out["status"])

    def last_launches(self) -> List[dict]:
        """rcpsp_last_launches: the launch classes of the last search call."""
        buf = (LaunchInfo * 16)()
        cnt = C.c_int32(0)
        self._check(self.lib.rcpsp_last_launches(self.ctx, buf, 16, C.byref(cnt)))
        return [{f: getattr(buf[k], f) for f, _ in LaunchInfo._fields_} for k in range(min(cnt.value, 16))]

    def kernel_launches(self) -> int:
        n = C.c_int64(0)
        self._check(self.lib.rcpsp_kernel_launches(self.ctx, C.byref(n)))
        return n.value

    def trace(self, id_: int, iterations: int) -> np.ndarray:
        buf = np.zeros(max(1, 3 * iterations), np.int32)
        written = C.c_int32(0)
        self._check(self.lib.rcpsp_get_trace(self.ctx, int(id_), _ptr(buf), buf.size, C.byref(written)))
        return buf[:3 * written.value].reshape(-1, 3)

    def evaluate_lists(self, id_: int, lists, mode: int = EVAL_AUTO, stream=None):
        lists = _i32(lists)
        n = self.n_of[int(id_)]
        cnt = lists.size // n
        start = np.zeros(cnt * n, np.int32)
        cmax = np.zeros(cnt, np.int32)
        work = np.zeros(cnt, np.int64)
        handle = getattr(stream, "cuda_stream", stream) or None
        self._check(self.lib.rcpsp_evaluate_lists(self.ctx, int(id_), _ptr(lists), cnt, mode, _ptr(start),
                                                  _ptr(cmax), _ptr(work, C.c_int64), handle))
        return cmax, start.reshape(cnt, n), work


class Server:
    """Continuous-batching solve server (rcpsp_server_* in include/rcpsp.h)."""

    def __init__(self, device: int = 0, slots: int = 8, max_batch: int = 256, memory_budget: int = 1 << 30,
                 poll_us: int = 100, lib_path: Optional[str] = None, slice_iterations: int = 0,
                 max_pending: int = 0):
        self.lib = library(lib_path)
        self.srv = C.c_void_p()
        cfg = ServerConfig(slots, max_batch, memory_budget, poll_us, slice_iterations, max_pending)
        rc = self.lib.rcpsp_server_create(C.byref(self.srv), device, C.byref(cfg))
        if rc != 0:
            raise RcpspError(rc, "server create")
        self.max_pending = max_pending
        self._buf = (Completion * 4096)()

    def submit(self, inst, tag: int, iterations: int = 1000, delta: int = 0, tabu_len: int = 0,
               mode: int = EVAL_AUTO, stop_at_cp: bool = True, level_key=None) -> bool:
        """Queues one request; False when the server's pending queue is full
        (max_pending), an error for anything else."""
        m = _Marshalled(inst, level_key)
        p = Params(iterations, delta, tabu_len, mode, int(stop_at_cp), 0, 0, 0, 0, 0)
        rc = self.lib.rcpsp_server_submit(self.srv, C.byref(m.s), C.byref(p), int(tag))
        if rc == E_TOO_LARGE and self.max_pending > 0:
            return False
        if rc != 0:
            raise RcpspError(rc, "submit")
        return True

    def poll(self, wait_ms: int = 0, capacity: int = 4096) -> List[dict]:
        cnt = C.c_int32(0)
        rc = self.lib.rcpsp_server_poll(self.srv, self._buf, min(capacity, 4096), C.byref(cnt), wait_ms)
        if rc != 0:
            raise RcpspError(rc, "poll")
        out = []
        for k in range(cnt.value):
            c = self._buf[k]
            n = c.n
            W = np.ctypeslib.as_array(c.order, (n,)).copy() if c.order else np.zeros(0, np.int32)
            S = np.ctypeslib.as_array(c.start, (n,)).copy() if c.start else np.zeros(0, np.int32)
            out.append(dict(tag=c.tag, status=c.status, best_cmax=c.best_cmax, iterations=c.iterations,
                            mode=c.eval_mode, cp=c.critical_path, evaluated=c.evaluated, work=c.work,
                            best_W=W, best_S=S, t_submit_ns=c.t_submit_ns, t_launch_ns=c.t_launch_ns,
                            t_done_ns=c.t_done_ns))
        return out

    def stats(self) -> dict:
        st = ServerStats()
        self.lib.rcpsp_server_get_stats(self.srv, C.byref(st))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.srv:
            self.lib.rcpsp_server_destroy(self.srv)
            self.srv = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
