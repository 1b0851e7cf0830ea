#!/usr/bin/env python
"""Throughput of the GB300 tabu search: evaluated neighbour schedules per second.

One step = one pass of the whole search path over a batch of synthetic
instances, replayed from one CUDA graph.  The line is quoted on the largest
single-GPU batch, the uneven one: 1024 instances with n uniform in
{30, 60, 90, 120, 300} activities, 4-8 resources, durations 1-50, 1000 tabu
iterations each (swap distance / tabu list by size), evaluator by the
selection rule, one persistent launch per launch class on forked streams.
``value`` counts the neighbour schedules the searches decoded (the paper's
Sched_sec) per second of device time with the instances resident in HBM;
``e2e`` is the same count through the C interface with host buffers
(instance upload, host preparation, search, result download).

Beside it, ``configs`` holds the two uniform batches with their own timing
and roofline -- 480 x n=30 (1000 iterations, swap distance 20, tabu list
60; also against one instance per launch) and 600 x n=120 (5000 iterations,
swap distance 60, tabu list 800) -- and ``serving`` the request stream at
2000 req/s and a second one at 0.8 x the rate the first one completed.

The roofline counts the work the kernel performed (the decoders' own
counters: placements, Alg. 5 / Alg. 4 loop steps, Alg. 6 update steps or
Eq. 7 reads, successor pushes, kept-state words; positions restored from
kept states are not counted) in word operations and shared-memory bytes,
against the integer-ALU rate and shared-memory bandwidth measured in the
same run by rcpsp_measure_peaks.

Run: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
     [--workload mixed_batch|j120_batch|j30_batch] [--iterations I]
Under torchrun each rank solves its own batch (weak scaling); with
--shard lpt the ranks split one batch by estimated cost instead and rank 0
gathers the results (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "mixed_batch": dict(family="mixed_batch", count=1024, iterations=1000, delta=0, tabu_len=0,
                        text="mixed_batch: 1024 synthetic RCPSP instances, n uniform in {30,60,90,120,300}, M in "
                             "4-8, durations 1-50, demands 1-10 w.p. 0.5, NC in {1.5,1.8,2.1}, RS in "
                             "{0.2,0.5,0.7,1.0}; 1000 tabu iterations each, swap distance / tabu list by size "
                             "(20/60, 60/250, 60/600, 60/800, 60/800), evaluator by the selection rule; one "
                             "CUDA-graph replay per step (one persistent launch per launch class, forked streams)"),
    "j120_batch": dict(family="j120_batch", count=600, iterations=5000, delta=60, tabu_len=800,
                       text="j120_batch: 600 synthetic RCPSP instances, n=120, M=4, durations 1-10, NC in "
                            "{1.5,1.8,2.1}, RS in {0.1,0.2,0.5,0.7,1.0}; 5000 tabu iterations each, swap distance "
                            "60, tabu list 800 (Table 2), evaluator by the selection rule; one CUDA-graph replay "
                            "per step"),
    "j30_batch": dict(family="j30_batch", count=480, iterations=1000, delta=20, tabu_len=60,
                      text="j30_batch: 480 synthetic RCPSP instances, n=30 (+2 dummies), M=4, durations 1-10, "
                           "demands 1-10 w.p. 0.5, NC in {1.5,1.8,2.1}, RS in {0.2,0.5,0.7,1.0}; 1000 tabu "
                           "iterations each, swap distance 20, tabu list 60, evaluator by the selection rule; "
                           "one persistent CUDA-graph launch per step"),
}
DEFAULT_WORKLOAD = "mixed_batch"
WORKLOAD = dict(WORKLOADS[DEFAULT_WORKLOAD])
WORKLOAD["name"] = DEFAULT_WORKLOAD
METRIC = "neighbour schedules evaluated/sec on 1 GB300 (bit-exact) + p50/p99 solve latency"
UNIT = "schedules/s"
KERNEL_SOURCES = ["paper_1711_04556_gb300/csrc/search_kernel.cuh", "paper_1711_04556_gb300/csrc/search_kernel.cu",
                  "paper_1711_04556_gb300/csrc/search_kernel_wide.cu",
                  "paper_1711_04556_gb300/csrc/search_kernel_solo.cu",
                  "paper_1711_04556_gb300/csrc/device_search.cuh",
                  "paper_1711_04556_gb300/csrc/rcpsp_internal.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "search_kernel_mixed_batch.traffic.json")
TUNE_TABLE = os.path.join(ROOT, "paper_1711_04556_gb300", "tune_shapes.tsv")
EVAL_TIME = 1


def workload_config(W, extra=None):
    cfg = {"workload": W["text"], "instances": W["count"], "iterations": W["iterations"],
           "delta": W["delta"] or "by size", "tabu_len": W["tabu_len"] or "by size",
           "l2": "flushed between timed steps (256 MiB write); inputs are a few MB, resident in HBM"}
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def words_per_step(inst) -> int:
    """32-bit words per time step of the packed profile: 4 resources of 8 bits
    per word when every capacity is below 128, else 2 of 16 bits."""
    fields = 4 if int(inst.cap.max()) <= 127 else 2
    w = -(-inst.m // fields)
    return 1 if w <= 1 else (2 if w <= 2 else 4)


def performed_work(insts, results):
    """Work the decodes performed, from the kernel's counters.

    Word operations (the resource words of the decoders, as the roofline
    counts them): time-indexed, every Alg. 5 step tests the step's profile
    words, every Alg. 6 step updates them, and every placement pushes its
    finish to its successors; capacity-indexed, one read per used resource
    (Eq. 7), one entry per Alg. 4 step, the successor pushes.  Shared-memory
    bytes: the same words at 4 bytes, Alg. 6 and Alg. 4 steps and pushes
    read and write, and every placement reads its earliest start.  Kept-state
    bytes: the decoder states of the current list written and read (global
    memory, L2-resident).  Positions restored from kept states are not
    counted: the kernel did not place them again.
    """
    ops = smem = kept = placed = 0
    for x, r in zip(insts, results):
        if r["mode"] == EVAL_TIME:
            wps = words_per_step(x)
            ops += r["succ_pushes"] + wps * (r["steps_done"] + r["update_units"])
            smem += 4 * (wps * (r["steps_done"] + 2 * r["update_units"]) + r["placements"] + 2 * r["succ_pushes"])
        else:
            ops += r["succ_pushes"] + r["update_units"] + r["steps_done"]
            smem += 4 * (r["update_units"] + 2 * r["steps_done"] + r["placements"] + 2 * r["succ_pushes"])
        kept += 4 * r["kept_words"]
        placed += r["placements"]
    return {"word_ops": ops, "smem_bytes": smem, "kept_state_bytes": kept, "placements": placed}


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def load_counters(path=TRAFFIC_FILE):
    """The committed ncu figures of the search kernel on this workload, if
    they were taken on the kernel source as it is now (else None)."""
    try:
        d = json.load(open(path))
        if d.get("kernel_hash") == kernel_hash():
            return d
    except Exception:
        pass
    return None


def roofline(work, per_step_s, peaks, counters):
    """The search kernel's roofline from the work it performed per step
    (all launches of a step; the launch classes run side by side on forked
    streams and the step's device time brackets them) against the peaks
    measured in this run."""
    alu_peak = peaks["int32_ops_per_s"] / 1e9 if peaks else None
    smem_peak = peaks["smem_bytes_per_s"] / 1e9 if peaks else None
    achieved = work["word_ops"] / per_step_s / 1e9
    smem_gbs = work["smem_bytes"] / per_step_s / 1e9
    basis = ("measured in this run by rcpsp_measure_peaks (best of 5 CUDA-event-timed launches, burst): "
             "32-bit integer ALU ops and conflict-free 16-byte shared-memory loads over all SMs")
    return {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Gop/s",
            "frac": achieved / alu_peak if alu_peak else None,
            "traffic": counters["dram_bytes_per_launch"] if counters else None,
            "ops_per_launch": work["word_ops"], "peak_basis": basis,
            "what": "word operations the decodes performed (kernel counters; kept-state positions excluded) over "
                    "the step's device time",
            "smem": {"bytes_per_launch": work["smem_bytes"], "achieved_gbs": smem_gbs, "peak_gbs": smem_peak,
                     "frac": smem_gbs / smem_peak if smem_peak else None,
                     "basis": "least shared-memory bytes of the performed decode work, against the measured "
                              "shared-memory load bandwidth"},
            "kept_state": {"bytes_per_launch": work["kept_state_bytes"],
                           "achieved_gbs": work["kept_state_bytes"] / per_step_s / 1e9,
                           "what": "kept decoder states written and read (global memory, L2-resident)"}}


def oracle_params(O, I, W, insts, iterations):
    """Per-instance oracle parameters; swap distance and tabu length 0 mean
    "by instance size", as the library reads them."""
    out = []
    for x in insts:
        d, t = (W["delta"], W["tabu_len"]) if W["delta"] else I.search_params(x.n - 2)
        out.append((iterations, d, t, O.AUTO, 1))
    return out


def cpu_baseline(W, sample: int, iterations: int, single: int, single_iterations: int):
    """The CPU reference, as it stands, on a bounded sample of the workload."""
    from oracle import oracle as O
    from paper_1711_04556_gb300 import instances as I
    O.build()
    insts = I.config_batch(W["family"], sample)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = O.tabu_search_batch(insts, oracle_params(O, I, W, insts, iterations), cores)
    dt = time.perf_counter() - t0
    ev = sum(r["evaluated"] for r in res)
    one = insts[:max(1, min(len(insts), single))]
    t1 = time.perf_counter()
    res1 = O.tabu_search_batch(one, oracle_params(O, I, W, one, single_iterations), 1)
    dt1 = time.perf_counter() - t1
    ev1 = sum(r["evaluated"] for r in res1)
    return {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {sample} of the {W['count']} instances, {iterations} iterations each "
                      f"(not the step's {W['iterations']}), one search per host thread ({ev} schedules in "
                      f"{dt:.2f} s)",
            "single_core": {"value": ev1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"first {len(one)} instances, {single_iterations} iterations each "
                                      f"({ev1} schedules in {dt1:.2f} s)"}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1711_04556_gb300 import instances as I
    O.build()
    W = WORKLOAD
    sample = args.reference_sample
    iters = args.reference_iterations or W["iterations"]
    insts = I.config_batch(W["family"], sample)
    cores = os.cpu_count() or 1
    params = oracle_params(O, I, W, insts, iters)
    for _ in range(args.warmup):
        O.tabu_search_batch(insts[:max(1, cores)], params[:max(1, cores)], cores)
    ev_total, t_total = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = O.tabu_search_batch(insts, params, cores)
        t_total += time.perf_counter() - t0
        ev_total += sum(r["evaluated"] for r in res)
    value = ev_total / t_total
    sample_txt = (f"each step: first {sample} of the {W['count']} instances, {iters} iterations each, one search "
                  f"per host thread")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(W, {"reference_sample": sample, "reference_iterations": iters}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_txt},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def percentiles(xs):
    xs = np.asarray(xs, dtype=np.float64)
    return float(np.percentile(xs, 50)), float(np.percentile(xs, 99))


def serving_stream(R, I, device, family, rate, seconds, iterations, pool_size=512, seed=5, drain_s=30.0,
                   max_pending=0, slice_iterations=0):
    """Poisson arrivals at `rate` req/s for `seconds` into a fresh
    continuous-batching server, measured from the stream's first request
    (the server is created, and pre-sized, before the stream starts).

    Requests cycle through a pool of distinct instances of `family`; each is
    one search of `iterations` iterations.  Latency = host time from submit
    to the completion record.  Submissions the server refuses because its
    pending queue is full (max_pending) count as rejected; requests still in
    flight `drain_s` after the last arrival count as not completed.
    """
    pool = I.config_batch(family, pool_size)
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, int(rate * seconds * 1.5) + 16))
    arrivals = arrivals[arrivals < seconds]
    done, accepted, rejected = [], 0, 0
    with R.Server(device, slots=12, max_batch=256, memory_budget=2 << 30, max_pending=max_pending,
                  slice_iterations=slice_iterations) as srv:
        t0 = time.perf_counter()
        k = 0
        while True:
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                if srv.submit(pool[k % pool_size], tag=k, iterations=iterations):
                    accepted += 1
                else:
                    rejected += 1
                k += 1
            done += srv.poll(wait_ms=0)
            if k == len(arrivals) and (len(done) == accepted or now > seconds + drain_s):
                break
            nxt = arrivals[k] - now if k < len(arrivals) else 0.002
            time.sleep(min(max(nxt, 0.0), 0.002))
        wall = time.perf_counter() - t0
        st = srv.stats()
    ok = [c for c in done if c["status"] == 0]
    lat = [(c["t_done_ns"] - c["t_submit_ns"]) / 1e6 for c in ok]
    ev = sum(c["evaluated"] for c in ok)
    p50, p99 = percentiles(lat) if lat else (None, None)
    return {"workload": f"{family} requests, {iterations} iterations each, Poisson {rate:.0f} req/s for "
                        f"{seconds:g} s, measured from the stream's first request"
                        + (f", time-sliced every {slice_iterations} iterations" if slice_iterations else ""),
            "offered_req_s": len(arrivals) / seconds, "submitted": int(len(arrivals)), "accepted": accepted,
            "rejected_queue_full": rejected, "completed": len(ok),
            "completed_req_s": len(ok) / wall, "schedules_per_s": ev / wall, "wall_s": wall,
            "latency_ms": {"p50": p50, "p90": float(np.percentile(lat, 90)) if lat else None, "p99": p99,
                           "max": float(max(lat)) if lat else None},
            "batches": st["batches"], "max_inflight_bytes": st["max_inflight_bytes"], "requeued": st["requeued"],
            "max_pending": max_pending}


def serving_run(R, I, device, args):
    """Config 5: the request stream at its offered rate (more than one GPU
    completes, so the pending queue is bounded and the excess shed), then a
    second stream at 0.8 x the rate the first completed, whose p50/p99 is
    the latency of a loaded but not overloaded server."""
    over = serving_stream(R, I, device, args.serving_family, args.serving_rate, args.serving_seconds,
                          args.serving_iterations, drain_s=args.serving_drain, max_pending=args.serving_max_pending,
                          slice_iterations=args.serving_slice)
    rate2 = max(1.0, 0.8 * over["completed_req_s"])
    under = serving_stream(R, I, device, args.serving_family, rate2, args.serving_seconds2,
                           args.serving_iterations, seed=6, drain_s=max(60.0, args.serving_drain),
                           slice_iterations=args.serving_slice)
    return {"offered_load": over, "at_0.8_completed_rate": under}


def coop_run(solver, I, insts, ids, ref_res, kw, st, args):
    """Co-operating searches (Sec. 6.1) of the same instances with the same
    total iterations per instance: B blocks of I/B iterations each, |F| = 16,
    Phi_max = 3, Phi_steps = 20 (Table 2).  Reports decoded schedules per
    second of device time and the mean best makespan beside that of the
    independent searches of the main measurement."""
    import torch
    B = args.coop_blocks
    it_block = max(1, kw["iterations"] // B)
    keys, words = [], []
    for k, x in enumerate(insts):
        kk, ww = I.coop_inputs(x, 1000 + k, 16, B, 256)
        keys.append(kk)
        words.append(ww)
    ckw = dict(iterations=it_block, delta=kw["delta"], tabu_len=kw["tabu_len"], mode=kw["mode"], blocks=B,
               working_set=16, phi_max=3, phi_steps=20, slot_keys=keys, words=words, stream=st)
    solver.coop_search(ids, **ckw)
    first = solver.results(ids)
    times = []
    for _ in range(args.coop_reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        solver.coop_search(ids, **ckw)
        e1.record(st)
        res = solver.results(ids)
        times.append(e0.elapsed_time(e1) / 1000.0)
        assert [r["best_cmax"] for r in res] == [r["best_cmax"] for r in first]
    ev = sum(r["evaluated"] for r in res)
    t = statistics.median(times)
    return {"what": f"{B} co-operating searches of {it_block} iterations per instance, working set 16, "
                    f"Phi_max 3, Phi_steps 20; the same instances as the main step",
            "schedules_per_s": ev / t, "ms_per_step": 1000 * t, "schedules_per_step": ev,
            "mean_best_cmax": float(np.mean([r["best_cmax"] for r in res])),
            "mean_best_cmax_independent": float(np.mean([r["best_cmax"] for r in ref_res])),
            "mean_cp_dev_pct": float(np.mean([100.0 * (r["best_cmax"] - r["cp"]) / r["cp"]
                                              for r in res if r["cp"] > 0])),
            "better_instances": int(sum(a["best_cmax"] < b["best_cmax"] for a, b in zip(res, ref_res))),
            "worse_instances": int(sum(a["best_cmax"] > b["best_cmax"] for a, b in zip(res, ref_res)))}


def search_kwargs(W, args, R):
    return dict(iterations=W["iterations"], delta=W["delta"], tabu_len=W["tabu_len"], mode=R.EVAL_AUTO,
                group_size=args.group_size, warps_per_cta=args.warps, cluster_size=args.cluster_size)


def shapes(solver, ids, W, args, R, st):
    """Launch shapes: the command line's, else the table of measured shapes
    (the committed output of rcpsp_autotune on this kind of GPU, read by
    every context through RCPSP_TUNE_CACHE) when it has every launch class
    of the batch, else rcpsp_autotune now (it adds them to the table)."""
    if args.group_size or args.warps or args.cluster_size:
        return "command line"
    if not args.retune:
        # a one-iteration search shows where the shape of every class comes from
        solver.search(ids, iterations=1, delta=W["delta"], tabu_len=W["tabu_len"], mode=R.EVAL_AUTO, stream=st)
        solver.results(ids)
        if all(c["shape_source"] == 1 for c in solver.last_launches()):
            return "table of shapes measured by rcpsp_autotune (" + os.path.relpath(TUNE_TABLE, ROOT) + ")"
    solver.autotune(ids, iterations=W["iterations"], delta=W["delta"], tabu_len=W["tabu_len"], mode=R.EVAL_AUTO,
                    trial_iterations=args.tune_iterations, stream=st)
    return f"rcpsp_autotune in this run ({args.tune_iterations} trial iterations)"


def measure_batch(solver, R, W, insts, args, st, flush, steps, warmup, sampler_gpu=None, world=1, dist=None):
    """Warm-up, then `steps` timed graph replays of the batch with an L2 flush
    before each; returns the measurement and the first results."""
    import torch
    ids = solver.load(insts)
    kw = search_kwargs(W, args, R)
    chosen = shapes(solver, ids, W, args, R, st)
    for _ in range(warmup):
        solver.search(ids, use_graph=True, stream=st, **kw)
        solver.results(ids)
    ref = solver.results(ids)
    assert all(r["status"] == 0 for r in ref), "a search reported an error"
    plan = solver.last_launches()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    barrier()
    sampler = ClockSampler(sampler_gpu) if sampler_gpu is not None else None
    if sampler:
        time.sleep(0.3)
    events = []
    k0 = solver.kernel_launches()
    t_wall = time.perf_counter()
    for _ in range(steps):
        with torch.cuda.stream(st):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        solver.search(ids, use_graph=True, stream=st, **kw)
        e1.record(st)
        events.append((e0, e1))
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = solver.kernel_launches() - k0
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in events]
    res = solver.results(ids)
    for a, b in zip(res, ref):   # every step reproduces the same searches
        assert a["best_cmax"] == b["best_cmax"] and a["evaluated"] == b["evaluated"] and a["work"] == b["work"]
    ev_step = sum(r["evaluated"] for r in ref)
    t0 = min(r["t_start_ns"] for r in res)
    done_ms = [(r["t_end_ns"] - t0) / 1e6 for r in res]
    service_ms = [(r["t_end_ns"] - r["t_start_ns"]) / 1e6 for r in res]
    b50, b99 = percentiles(done_ms)
    s50, s99 = percentiles(service_ms)
    return {"ids": ids, "ref": ref, "kw": kw, "step_ms": step_ms, "ev_step": ev_step, "launches": launches,
            "clocks": clocks, "wall_s": t_wall, "plan": plan, "chosen": chosen,
            "latency": {"in_batch_completion": {"p50": b50, "p99": b99,
                                                "what": "device time from the first search start to each "
                                                        "instance's results, one batched step"},
                        "in_batch_service": {"p50": s50, "p99": s99,
                                             "what": "device time from each search start to its results"}}}


def sub_config(solver, R, I, name, args, st, flush, peaks):
    """One of the uniform batches on its own: value, step time, roofline."""
    W = dict(WORKLOADS[name])
    insts = I.config_batch(W["family"], W["count"])
    steps = args.j30_steps if name == "j30_batch" else args.j120_steps
    m = measure_batch(solver, R, W, insts, args, st, flush, steps, 3)
    per_step = sum(m["step_ms"]) / 1000.0 / steps
    work = performed_work(insts, m["ref"])
    out = {"config": workload_config(W), "value": m["ev_step"] / per_step, "unit": UNIT,
           "ms_per_step": 1000 * per_step, "steps": steps, "warmup": 3, "schedules_per_step": m["ev_step"],
           "gpu_launches": m["launches"], "launch_classes": m["plan"], "shapes_from": m["chosen"],
           "roofline": roofline(work, per_step, peaks, None), "latency_ms": m["latency"],
           "placements_per_neighbour": work["placements"] / max(1, m["ev_step"])}
    if name == "j30_batch" and args.plain_sample > 0:
        out["plain_per_instance_launch"] = plain_run(solver, m["ids"], m["kw"], st, args.plain_sample,
                                                     out["value"])
    solver.free(m["ids"])
    return out


def plain_run(solver, ids, kw, st, sample, batched_value):
    """The plain form: one instance per launch, sequential, on a sample."""
    import torch
    sid = ids[:sample]
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in sid:
        solver.search([i], use_graph=False, stream=st, **kw)
    e1.record(st)
    torch.cuda.synchronize()
    ev = sum(r["evaluated"] for r in solver.results(sid))
    plain = ev / (e0.elapsed_time(e1) / 1000.0)
    return {"value": plain, "unit": UNIT, "sample": f"first {len(sid)} instances, one launch each",
            "batched_over_plain": batched_value / plain}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the benchmark needs a GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1711_04556_gb300 import build as B
    from paper_1711_04556_gb300 import instances as I
    from paper_1711_04556_gb300 import rcpsp as R
    B.build()
    from paper_1711_04556_gb300 import replicas
    # the committed shape table, through a copy that the autotuner may rewrite
    tune_copy = None
    if os.path.exists(TUNE_TABLE) and "RCPSP_TUNE_CACHE" not in os.environ:
        fd, tune_copy = tempfile.mkstemp(suffix=".tsv")
        os.close(fd)
        shutil.copyfile(TUNE_TABLE, tune_copy)
        os.environ["RCPSP_TUNE_CACHE"] = tune_copy
    W = WORKLOAD
    if args.shard == "lpt":
        # one batch split over the ranks by estimated cost (strong scaling)
        batch = I.config_batch(W["family"], W["count"])
        if len(batch) < world:
            raise RuntimeError("fewer instances than ranks")
        parts = replicas.lpt_partition([replicas.estimated_cost(x, W["iterations"], W["delta"]) for x in batch],
                                       world)
        insts = [batch[i] for i in parts[rank]]
    else:
        parts = None
        insts = replicas.shard(W["family"], W["count"], rank)
    peaks = R.measure_peaks(local)
    solver = R.Solver(local)
    st = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)   # 256 MiB > L2

    # ---------------- timed region: K steps, device time by CUDA events
    m = measure_batch(solver, R, W, insts, args, st, flush, args.steps, args.warmup, sampler_gpu=local, world=world,
                      dist=dist)
    ids, ref_res, kw = m["ids"], m["ref"], m["kw"]
    dev_s, ev_all = replicas.reduce_timing(dist, dev, sum(m["step_ms"]) / 1000.0, float(m["ev_step"]), world)
    value = ev_all * args.steps / dev_s

    # ---------------- end to end through the C interface, host buffers
    h0, d0 = solver.transfer_bytes()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_e2e = time.perf_counter()
    ev_e2e = 0
    # a client that loads the next batch while the current one is searched:
    # every step still uploads its instances and reads its results back
    nxt = solver.load(insts)
    for k in range(e2e_steps):
        ids2 = nxt
        solver.search(ids2, use_graph=False, stream=st, **kw)
        if k + 1 < e2e_steps:
            nxt = solver.load(insts)
        out = solver.results(ids2)
        ev_e2e += sum(r["evaluated"] for r in out)
        solver.free(ids2)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_e2e = time.perf_counter() - t_e2e
    h1, d1 = solver.transfer_bytes()
    t_e2e_max, ev_e2e_all = replicas.reduce_timing(dist, dev, t_e2e, float(ev_e2e), world)
    e2e_val = ev_e2e_all / t_e2e_max
    all_res = (replicas.gather_results(dist, ref_res, parts[rank], W["count"], world, rank)
               if parts is not None else None)
    if rank != 0:
        solver.close()
        if world > 1:
            dist.destroy_process_group()
        return 0

    per_step_s = dev_s / args.steps if world == 1 else sum(m["step_ms"]) / 1000.0 / args.steps
    work = performed_work(insts, ref_res)
    counters = load_counters() if W["name"] == DEFAULT_WORKLOAD and parts is None else None
    extra = {}
    if world == 1:
        # the uniform batches, each measured on its own
        if not args.no_subconfigs:
            extra["configs"] = {name: sub_config(solver, R, I, name, args, st, flush, peaks)
                                for name in ("j30_batch", "j120_batch") if name != W["name"]}
        # single-instance solve latency (one instance, 100 iterations), repeated
        one = I.config_batch("j30_single")
        lat = []
        for _ in range(args.latency_reps):
            t0h = time.perf_counter()
            i1 = solver.load(one)
            solver.search(i1, iterations=100, delta=20, tabu_len=60, mode=R.EVAL_AUTO, stream=st)
            solver.results(i1)
            solver.free(i1)
            lat.append((time.perf_counter() - t0h) * 1000)
        latency = dict(m["latency"])
        if lat:
            p50, p99 = percentiles(lat)
            latency["single_instance_e2e"] = {"p50": p50, "p99": p99, "reps": args.latency_reps,
                                              "what": "1 instance, 100 iterations, load+search+results through "
                                                      "the C API"}
        extra["latency_ms"] = latency
        if args.coop_blocks > 0:
            extra["cooperation"] = coop_run(solver, I, insts, ids, ref_res, kw, st, args)
        if args.serving_seconds > 0:
            extra["serving"] = serving_run(R, I, local, args)
    qres = all_res if all_res is not None else ref_res
    devs = [100.0 * (r["best_cmax"] - r["cp"]) / r["cp"] for r in qres if r["cp"] > 0]
    extra["quality"] = {"mean_cp_dev_pct": float(np.mean(devs)) if devs else None,
                        "at_critical_path": int(sum(r["best_cmax"] == r["cp"] for r in qres)),
                        "instances": len(qres)}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(W, args.cpu_sample, args.cpu_iterations, args.cpu_single, args.cpu_single_iterations)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(m["step_ms"]) / args.steps, "higher_is_better": True,
        "scaling": "strong" if parts is not None else "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": workload_config(W, {
            "parallelism": (f"lpt{world}" if parts is not None else f"replicas{world}") if world > 1 else "single GPU",
            "schedules_per_step": m["ev_step"], "wall_s_timed": m["wall_s"], "launch_classes": m["plan"],
            "shapes_from": m["chosen"], "placements_per_neighbour": work["placements"] / max(1, m["ev_step"])}),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": (h1 - h0) // e2e_steps,
                "d2h_bytes_per_step": (d1 - d0) // e2e_steps, "steps": e2e_steps},
        "gpu_launches": m["launches"],
        "roofline": roofline(work, per_step_s, peaks, counters),
        "cpu_baseline": cpu,
        "clocks": m["clocks"],
        "peaks": peaks,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    solver.close()
    if tune_copy:
        os.unlink(tune_copy)
    if world > 1:
        dist.destroy_process_group()
    return 0


def set_workload(name: str, iterations: int) -> None:
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[name])
    WORKLOAD["name"] = name
    if iterations:
        WORKLOAD["iterations"] = iterations
        WORKLOAD["text"] = WORKLOAD["text"].replace(f"{WORKLOADS[name]['iterations']} tabu iterations",
                                                    f"{iterations} tabu iterations")


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD,
                    help="instance batch of one step (the bench line is quoted on mixed_batch)")
    ap.add_argument("--iterations", type=int, default=0, help="tabu iterations per instance (0: the workload's)")
    ap.add_argument("--group-size", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--cluster-size", type=int, default=0)
    ap.add_argument("--retune", action="store_true", help="run rcpsp_autotune even when the shape table has the GPU")
    ap.add_argument("--tune-iterations", type=int, default=48)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-subconfigs", action="store_true", help="skip the j30 and j120 measurements")
    ap.add_argument("--j30-steps", type=int, default=20)
    ap.add_argument("--j120-steps", type=int, default=3)
    ap.add_argument("--serving-seconds", type=float, default=60.0)
    ap.add_argument("--serving-seconds2", type=float, default=30.0,
                    help="length of the second stream (0.8 x the completed rate)")
    ap.add_argument("--serving-rate", type=float, default=2000.0)
    ap.add_argument("--serving-family", default="mixed_batch")
    ap.add_argument("--serving-iterations", type=int, default=1000)
    ap.add_argument("--serving-drain", type=float, default=10.0)
    ap.add_argument("--serving-max-pending", type=int, default=4096)
    ap.add_argument("--serving-slice", type=int, default=0,
                    help="server time slice in iterations (0: no slicing)")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving measurement and print its JSON object")
    ap.add_argument("--plain-sample", type=int, default=48)
    ap.add_argument("--latency-reps", type=int, default=100)
    ap.add_argument("--cpu-sample", type=int, default=32, help="instances of the oracle's timed sample")
    ap.add_argument("--cpu-iterations", type=int, default=100, help="iterations per instance of that sample")
    ap.add_argument("--cpu-single", type=int, default=8, help="instances of the single-core sample")
    ap.add_argument("--cpu-single-iterations", type=int, default=20)
    ap.add_argument("--reference-sample", type=int, default=16)
    ap.add_argument("--reference-iterations", type=int, default=20,
                    help="iterations per instance of each reference step (0: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", choices=("seeds", "lpt"), default="seeds",
                    help="seeds: each rank its own batch (weak scaling); lpt: one batch split over the ranks "
                         "by estimated cost, results gathered on rank 0 (strong scaling)")
    ap.add_argument("--coop-blocks", type=int, default=4,
                    help="co-operating searches per instance in the cooperation measurement (0 skips it)")
    ap.add_argument("--coop-reps", type=int, default=1)
    args = ap.parse_args()
    set_workload(args.workload, args.iterations)
    if args.warmup < 3:
        args.warmup = 3
    if args.serving_only:
        import torch
        from paper_1711_04556_gb300 import build as B
        from paper_1711_04556_gb300 import instances as I
        from paper_1711_04556_gb300 import rcpsp as R
        B.build()
        torch.cuda.init()
        print(json.dumps({"serving": serving_run(R, I, 0, args)}), flush=True)
        return 0
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
