#!/usr/bin/env python
"""Throughput of the GB300 tabu search: evaluated neighbour schedules per second.

One step = one pass of the whole search path over a batch of synthetic
instances: 480 instances of 30 non-dummy activities (4 resources, network
complexity 1.5/1.8/2.1, resource strength 0.2/0.5/0.7/1.0), 1000 tabu
iterations each (swap distance 20, tabu list 60, evaluator by the selection
rule), all in one persistent launch replayed from a CUDA graph.  ``value``
counts the neighbour schedules the searches decoded (the paper's Sched_sec)
per second of device time with the instances resident in HBM; ``e2e`` is
the same count through the C interface with host buffers (instance upload,
host preparation, search, result download).

Run: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
     [--workload j30_batch|j120_batch|mixed_batch] [--iterations I]
Under torchrun each rank solves its own 480 instances (weak scaling); with
--shard lpt the ranks split one batch by estimated cost instead and rank 0
gathers the results (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "j30_batch": dict(family="j30_batch", count=480, iterations=1000, delta=20, tabu_len=60,
                      text="j30_batch: 480 synthetic RCPSP instances, n=30 (+2 dummies), M=4, durations 1-10, "
                           "demands 1-10 w.p. 0.5, NC in {1.5,1.8,2.1}, RS in {0.2,0.5,0.7,1.0}; 1000 tabu "
                           "iterations each, swap distance 20, tabu list 60, evaluator by the selection rule; "
                           "one persistent CUDA-graph launch per step"),
    "j120_batch": dict(family="j120_batch", count=600, iterations=5000, delta=60, tabu_len=800,
                       text="j120_batch: 600 synthetic RCPSP instances, n=120, M=4, durations 1-10, NC in "
                            "{1.5,1.8,2.1}, RS in {0.1,0.2,0.5,0.7,1.0}; 5000 tabu iterations each, swap distance "
                            "60, tabu list 800, evaluator by the selection rule; one CUDA-graph replay per step"),
    "mixed_batch": dict(family="mixed_batch", count=1024, iterations=1000, delta=0, tabu_len=0,
                        text="mixed_batch: 1024 synthetic RCPSP instances, n uniform in {30,60,90,120,300}, M in "
                             "4-8, durations 1-50; 1000 tabu iterations each, swap distance / tabu list by size "
                             "(20/60, 60/250, 60/600, 60/800, 60/800), evaluator by the selection rule; one "
                             "CUDA-graph replay per step (launch classes on forked streams)"),
}
WORKLOAD = dict(WORKLOADS["j30_batch"])
METRIC = "neighbour schedules evaluated/sec on 1 GB300 (bit-exact) + p50/p99 solve latency"
UNIT = "schedules/s"
KERNEL_SOURCES = ["paper_1711_04556_gb300/csrc/search_kernel.cuh", "paper_1711_04556_gb300/csrc/search_kernel.cu",
                  "paper_1711_04556_gb300/csrc/device_search.cuh",
                  "paper_1711_04556_gb300/csrc/rcpsp_internal.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "search_kernel_j30_batch.traffic.json")


def workload_config(extra=None):
    cfg = {"workload": WORKLOAD["text"],
           "instances": WORKLOAD["count"], "iterations": WORKLOAD["iterations"],
           "delta": WORKLOAD["delta"], "tabu_len": WORKLOAD["tabu_len"],
           "l2": "flushed between timed steps (256 MiB write); inputs are a few hundred KB"}
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


def algorithmic_ops(insts, results):
    """Resource-cell operations of the decodes the searches performed.

    Time-indexed (Algs. 5-7): every loop step of Alg. 5 tests M cells, Alg. 6
    updates M cells on each of the d_i steps of every activity (M * UB per
    schedule) and Alg. 7 reads |E| predecessor finish times.  Capacity-indexed
    (Eq. 7, Alg. 4): one read per used resource of every activity, one cell per
    Alg. 4 loop step, |E| predecessor reads.  ``work`` is the exact Alg. 5 or
    Alg. 4 step count the kernel reports (bit-exact with the CPU reference).
    """
    ops = 0
    for inst, r in zip(insts, results):
        ev = r["evaluated"]
        arcs = int(inst.succ_off[-1])
        if r["mode"] == 1:
            ops += inst.m * (r["work"] + ev * int(inst.dur.sum())) + ev * arcs
        else:
            used = int(np.count_nonzero(inst.req))
            ops += r["work"] + ev * (used + arcs)
    return ops


def algorithmic_smem_bytes(insts, results):
    """Shared-memory bytes the decodes need at the least, with the search
    state in shared memory in its packed form.  Time-indexed: every Alg. 5
    step reads the step's profile words (WPS words of 4 bytes: resources in
    8-bit fields, 16-bit when a capacity exceeds 127), and each of the d_i
    steps of Alg. 6 reads and writes them.  Capacity-indexed: one 4-byte read
    per used resource (Eq. 7), a read and a write per Alg. 4 loop step.  Both
    read the list (N words) and |E| finish times.  ``work`` and ``evaluated``
    are the kernel's exact counts."""
    total = 0
    for inst, r in zip(insts, results):
        ev = r["evaluated"]
        arcs = int(inst.succ_off[-1])
        if r["mode"] == 1:
            fields = 4 if int(inst.cap.max()) <= 127 else 2
            wps = -(-inst.m // fields)
            wps = 1 if wps <= 1 else (2 if wps <= 2 else 4)
            total += 4 * wps * (r["work"] + 2 * ev * int(inst.dur.sum()))
        else:
            used = int(np.count_nonzero(inst.req))
            total += 8 * r["work"] + 4 * ev * used
        total += 4 * ev * (inst.n + arcs)
    return total


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def load_counters():
    """The committed ncu figures of the search kernel, if they were taken on
    the kernel source as it is now (else None)."""
    try:
        d = json.load(open(TRAFFIC_FILE))
        if d.get("kernel_hash") == kernel_hash():
            return d
    except Exception:
        pass
    return None


def smem_roofline(counters, per_launch_s, sms, max_mhz):
    """Shared-memory side of the roofline: the captured launch's wavefronts
    over the live launch duration, against one 128-byte wavefront per SM per
    clock."""
    if not counters or not counters.get("smem_wavefronts_per_launch"):
        return None
    wf = counters["smem_wavefronts_per_launch"]
    peak = sms * max_mhz * 1e6
    return {"wavefronts_per_launch": wf, "achieved_per_s": wf / per_launch_s, "peak_per_s": peak,
            "frac": wf / per_launch_s / peak, "issue_active_pct": counters.get("issue_active_pct"),
            "alu_pipe_active_pct": counters.get("alu_pipe_active_pct"),
            "basis": "wavefronts from the committed ncu capture of this kernel source; peak = SMs x 1 wavefront "
                     "per clock (derived)"}


def oracle_params(O, I, insts, iterations):
    """Per-instance oracle parameters; swap distance and tabu length 0 mean
    "by instance size", as the library reads them."""
    out = []
    for x in insts:
        d, t = (WORKLOAD["delta"], WORKLOAD["tabu_len"]) if WORKLOAD["delta"] else I.search_params(x.n - 2)
        out.append((iterations, d, t, O.AUTO, 1))
    return out


def cpu_baseline(sample: int, iterations: int):
    """The CPU reference, as it stands, on a bounded sample of the workload."""
    from oracle import oracle as O
    from paper_1711_04556_gb300 import instances as I
    O.build()
    insts = I.config_batch(WORKLOAD["family"], sample)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = O.tabu_search_batch(insts, oracle_params(O, I, insts, iterations), cores)
    dt = time.perf_counter() - t0
    ev = sum(r["evaluated"] for r in res)
    # the same oracle on one host thread, on the first instances of the sample
    one = insts[:max(1, min(len(insts), 16))]
    t1 = time.perf_counter()
    res1 = O.tabu_search_batch(one, oracle_params(O, I, one, iterations), 1)
    dt1 = time.perf_counter() - t1
    ev1 = sum(r["evaluated"] for r in res1)
    return {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {sample} of the {WORKLOAD['count']} instances, {iterations} "
                      f"iterations each, one search per host thread ({ev} schedules in {dt:.2f} s)",
            "single_core": {"value": ev1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"first {len(one)} instances, {iterations} iterations each "
                                      f"({ev1} schedules in {dt1:.2f} s)"}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1711_04556_gb300 import instances as I
    O.build()
    sample = args.reference_sample
    insts = I.config_batch(WORKLOAD["family"], sample)
    cores = os.cpu_count() or 1
    params = oracle_params(O, I, insts, WORKLOAD["iterations"])
    for _ in range(args.warmup):
        O.tabu_search_batch(insts[:max(1, cores)], params[:max(1, cores)], cores)
    ev_total, t_total = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = O.tabu_search_batch(insts, params, cores)
        t_total += time.perf_counter() - t0
        ev_total += sum(r["evaluated"] for r in res)
    value = ev_total / t_total
    sample_txt = (f"each step: first {sample} of the {WORKLOAD['count']} instances, {WORKLOAD['iterations']} "
                  f"iterations each, one search per host thread")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference", "config": workload_config({"reference_sample": sample}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_txt},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_run(R, I, device, family, rate, seconds, iterations, pool_size=512, seed=5, drain_s=30.0,
                slice_iterations=0, warm_s=1.0):
    """Poisson arrivals at `rate` req/s for `warm_s` + `seconds` into the
    continuous-batching server; the first `warm_s` seconds bring the server
    and the GPU to their steady state and are not measured.

    Requests cycle through a pool of distinct instances of `family`; each is
    one search of `iterations` iterations.  Latency = host time from submit
    to the completion record.  Requests still in flight `drain_s` after the
    last arrival are counted as not completed.
    """
    pool = I.config_batch(family, pool_size)
    rng = np.random.default_rng(seed)
    total = warm_s + seconds
    gaps = rng.exponential(1.0 / rate, int(rate * total * 1.5) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < total]
    done = []
    with R.Server(device, slots=8, max_batch=256, memory_budget=2 << 30, slice_iterations=slice_iterations) as srv:
        # warm-up: batches on the slots (kernels loaded, staging allocated)
        # before the measured stream
        for k in range(64):
            srv.submit(pool[k % pool_size], tag=-1 - k, iterations=iterations)
            if k % 8 == 7:
                time.sleep(0.002)
        warm = 0
        t_w = time.perf_counter()
        while warm < 64 and time.perf_counter() - t_w < drain_s:
            warm += len(srv.poll(wait_ms=20))
        st0 = srv.stats()
        t0 = time.perf_counter()
        k = 0
        while True:
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                srv.submit(pool[k % pool_size], tag=k, iterations=iterations)
                k += 1
            done += srv.poll(wait_ms=0)
            if k == len(arrivals) and (len(done) == k or now > total + drain_s):
                break
            nxt = arrivals[k] - now if k < len(arrivals) else 0.002
            time.sleep(min(max(nxt, 0.0), 0.002))
        wall = time.perf_counter() - t0 - warm_s
        st = srv.stats()
    measured = [c for c in done if c["tag"] >= 0 and arrivals[c["tag"]] >= warm_s]
    n_meas = int(np.count_nonzero(arrivals >= warm_s))
    lat = [(c["t_done_ns"] - c["t_submit_ns"]) / 1e6 for c in measured if c["status"] == 0]
    ev = sum(c["evaluated"] for c in measured)
    st = {k: st[k] - st0[k] if k in ("batches",) else st[k] for k in st}
    p50, p99 = percentiles(lat) if lat else (None, None)
    p90 = float(np.percentile(lat, 90)) if lat else None
    lmax = float(max(lat)) if lat else None
    return {"workload": f"{family} requests, {iterations} iterations each, Poisson {rate:g} req/s for {seconds:g} s "
                        f"measured after {warm_s:g} s of the same stream (and 64 warm-up requests)"
                        + (f", time-sliced every {slice_iterations} iterations" if slice_iterations else ""),
            "requeued": st.get("requeued", 0),
            "offered_req_s": n_meas / seconds, "completed": len(lat), "submitted": n_meas,
            "completed_req_s": len(lat) / wall, "schedules_per_s": ev / wall, "wall_s": wall,
            "latency_ms": {"p50": p50, "p90": p90, "p99": p99, "max": lmax}, "batches": st["batches"],
            "max_inflight_bytes": st["max_inflight_bytes"]}


def coop_run(solver, R, I, insts, ids, ref_res, kw, st, args):
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
    for _ in range(2):
        solver.coop_search(ids, **ckw)
        first = solver.results(ids)
    times = []
    for _ in range(3):
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
    cm = float(np.mean([r["best_cmax"] for r in res]))
    ind = float(np.mean([r["best_cmax"] for r in ref_res]))
    return {"what": f"{B} co-operating searches of {it_block} iterations per instance, working set 16, "
                    f"Phi_max 3, Phi_steps 20; the same instances as the main step",
            "schedules_per_s": ev / t, "ms_per_step": 1000 * t, "schedules_per_step": ev,
            "mean_best_cmax": cm, "mean_best_cmax_independent": ind,
            "mean_cp_dev_pct": float(np.mean([100.0 * (r["best_cmax"] - r["cp"]) / r["cp"]
                                              for r in res if r["cp"] > 0])),
            "better_instances": int(sum(a["best_cmax"] < b["best_cmax"] for a, b in zip(res, ref_res))),
            "worse_instances": int(sum(a["best_cmax"] > b["best_cmax"] for a, b in zip(res, ref_res)))}


def percentiles(xs):
    xs = np.asarray(xs, dtype=np.float64)
    return float(np.percentile(xs, 50)), float(np.percentile(xs, 99))


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
    if args.shard == "lpt":
        # one batch split over the ranks by estimated cost (strong scaling)
        batch = I.config_batch(WORKLOAD["family"], WORKLOAD["count"])
        if len(batch) < world:
            raise RuntimeError("fewer instances than ranks")
        parts = replicas.lpt_partition([replicas.estimated_cost(x, WORKLOAD["iterations"], WORKLOAD["delta"])
                                        for x in batch], world)
        insts = [batch[i] for i in parts[rank]]
    else:
        parts = None
        insts = replicas.shard(WORKLOAD["family"], WORKLOAD["count"], rank)
    solver = R.Solver(local)
    st = torch.cuda.Stream(device=dev)
    kw = dict(iterations=WORKLOAD["iterations"], delta=WORKLOAD["delta"], tabu_len=WORKLOAD["tabu_len"],
              mode=R.EVAL_AUTO, group_size=args.group_size, warps_per_cta=args.warps,
              cluster_size=args.cluster_size)
    ids = solver.load(insts)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)   # 256 MiB > L2
    tuned = None
    if not (args.group_size or args.warps or args.cluster_size):
        tuned = solver.autotune(ids, iterations=kw["iterations"], delta=kw["delta"], tabu_len=kw["tabu_len"],
                                mode=R.EVAL_AUTO, trial_iterations=args.tune_iterations, stream=st)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        solver.search(ids, use_graph=True, stream=st, **kw)
        solver.results(ids)
    ref_res = solver.results(ids)
    assert all(r["status"] == 0 for r in ref_res), "a search reported an error"
    ev_step = sum(r["evaluated"] for r in ref_res)
    ops_step = algorithmic_ops(insts, ref_res)
    smem_bytes_step = algorithmic_smem_bytes(insts, ref_res)

    # ---------------- timed region: K steps, device time by CUDA events
    barrier()
    sampler = ClockSampler(local)
    time.sleep(0.3)
    events = []
    k0 = solver.kernel_launches()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
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
    launches_timed = solver.kernel_launches() - k0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in events]
    res = solver.results(ids)
    for a, b in zip(res, ref_res):   # every step reproduces the same searches
        assert a["best_cmax"] == b["best_cmax"] and a["evaluated"] == b["evaluated"]
    dev_s, ev_all = replicas.reduce_timing(dist, dev, sum(step_ms) / 1000.0, float(ev_step), world)
    value = ev_all * args.steps / dev_s

    # in-batch solve latency from the device timestamps of the last step
    t0 = min(r["t_start_ns"] for r in res)
    done_ms = [(r["t_end_ns"] - t0) / 1e6 for r in res]
    service_ms = [(r["t_end_ns"] - r["t_start_ns"]) / 1e6 for r in res]

    # ---------------- end to end through the C interface, host buffers
    h0, d0 = solver.transfer_bytes()
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
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
    barrier()
    t_e2e = time.perf_counter() - t_e2e
    h1, d1 = solver.transfer_bytes()
    t_e2e_max, ev_e2e_all = replicas.reduce_timing(dist, dev, t_e2e, float(ev_e2e), world)
    e2e_val = ev_e2e_all / t_e2e_max
    # the whole batch's results on rank 0 (after the timed regions)
    all_res = (replicas.gather_results(dist, ref_res, parts[rank], WORKLOAD["count"], world, rank)
               if parts is not None else None)

    extra = {}
    if rank == 0:
        # plain form: one instance per launch, sequential, on a sample
        sample = insts[:args.plain_sample]
        sid = ids[:args.plain_sample]
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ev_plain = 0
        for i in sid:
            solver.search([i], use_graph=False, stream=st, **kw)
        e1.record(st)
        barrier()
        ev_plain = sum(r["evaluated"] for r in solver.results(sid))
        plain = ev_plain / (e0.elapsed_time(e1) / 1000.0)
        extra["plain_per_instance_launch"] = {"value": plain, "unit": UNIT,
                                              "sample": f"first {len(sid)} instances, one launch each",
                                              "batched_over_plain": value / world / plain}
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
        p50, p99 = percentiles(lat)
        b50, b99 = percentiles(done_ms)
        s50, s99 = percentiles(service_ms)
        if args.coop_blocks > 0:
            extra["cooperation"] = coop_run(solver, R, I, insts, ids, ref_res, kw, st, args)
        if args.serving_seconds > 0:
            extra["serving"] = serving_run(R, I, local, args.serving_family, args.serving_rate, args.serving_seconds,
                                           args.serving_iterations, drain_s=args.serving_drain,
                                           slice_iterations=args.serving_slice)
        # solution quality: deviation of the best makespan from the critical-path
        # lower bound (the paper's "CP dev." measure), and how many reach it
        qres = all_res if all_res is not None else ref_res
        devs = [100.0 * (r["best_cmax"] - r["cp"]) / r["cp"] for r in qres if r["cp"] > 0]
        extra["quality"] = {"mean_cp_dev_pct": float(np.mean(devs)) if devs else None,
                            "at_critical_path": int(sum(r["best_cmax"] == r["cp"] for r in qres)),
                            "instances": len(qres)}
        extra["latency_ms"] = {
            "single_instance_e2e": {"p50": p50, "p99": p99, "reps": args.latency_reps,
                                    "what": "1 instance, 100 iterations, load+search+results through the C API"},
            "in_batch_completion": {"p50": b50, "p99": b99,
                                    "what": "device time from the first search start to each instance's results, "
                                            "one batched step"},
            "in_batch_service": {"p50": s50, "p99": s99, "what": "device time from each search start to its results"}}

    if rank != 0:
        solver.close()
        if world > 1:
            dist.destroy_process_group()
        return 0

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * 128 * max_mhz * 1e6 / 1e9            # INT32 lane-ops/s, in Gop/s
    per_launch_s = dev_s / args.steps if world == 1 else sum(step_ms) / 1000.0 / args.steps
    achieved = ops_step / per_launch_s / 1e9
    # the committed counters were taken on the j30 batch; its DRAM traffic does
    # not depend on the launch shape, the shared-memory wavefronts do
    counters = load_counters() if WORKLOAD["family"] == "j30_batch" else None
    shape = tuple(tuned or (args.group_size, args.warps, args.cluster_size or 1))
    smem = smem_roofline(counters, per_launch_s, sms, max_mhz) if shape == (4, 12, 1) else None
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample, args.cpu_iterations or WORKLOAD["iterations"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / args.steps, "higher_is_better": True,
        "scaling": "strong" if parts is not None else "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": workload_config({"parallelism": (f"lpt{world}" if parts is not None else f"replicas{world}")
                                   if world > 1 else "single GPU",
                                   "schedules_per_step": ev_step, "wall_s_timed": t_wall,
                                   "launch_shape": dict(zip(("group_size", "warps_per_cta", "cluster_size"),
                                                            tuned or (args.group_size, args.warps,
                                                                      args.cluster_size or 1)),
                                                        chosen_by="rcpsp_autotune" if tuned else "command line")}),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": (h1 - h0) // e2e_steps,
                "d2h_bytes_per_step": (d1 - d0) // e2e_steps},
        "gpu_launches": launches_timed,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                     "frac": achieved / peak, "traffic": counters["dram_bytes_per_launch"] if counters else None,
                     "ops_per_launch": ops_step,
                     "peak_basis": f"{sms} SMs x 128 INT32 lanes x {max_mhz:.0f} MHz (derived, not measured)",
                     "smem": smem,
                     "smem_algorithmic": {
                         "bytes_per_launch": smem_bytes_step,
                         "achieved_gbs": smem_bytes_step / per_launch_s / 1e9,
                         "peak_gbs": sms * 128 * max_mhz * 1e6 / 1e9,
                         "frac": smem_bytes_step / per_launch_s / (sms * 128 * max_mhz * 1e6),
                         "basis": "least shared-memory bytes of the decodes from the exact work counts; peak = "
                                  "SMs x 128 bytes per clock (derived)"},
                     **({} if WORKLOAD["family"] == "j30_batch" else
                        {"note": "ops count full decodes; where prefix reuse is on (several decode rounds per "
                                 "iteration) the kernel skips part of them, so this fraction overstates"})},
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def set_workload(name: str, iterations: int) -> None:
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[name])
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="j30_batch",
                    help="instance batch of one step (the bench line is quoted on j30_batch)")
    ap.add_argument("--iterations", type=int, default=0, help="tabu iterations per instance (0: the workload's)")
    ap.add_argument("--group-size", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--cluster-size", type=int, default=0)
    ap.add_argument("--tune-iterations", type=int, default=48)
    ap.add_argument("--serving-seconds", type=float, default=5.0)
    ap.add_argument("--serving-rate", type=float, default=2000.0)
    ap.add_argument("--serving-family", default=WORKLOAD["family"])
    ap.add_argument("--serving-iterations", type=int, default=WORKLOAD["iterations"])
    ap.add_argument("--serving-drain", type=float, default=30.0)
    ap.add_argument("--serving-slice", type=int, default=0,
                    help="server time slice in iterations (0: no slicing)")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving measurement and print its JSON object")
    ap.add_argument("--plain-sample", type=int, default=48)
    ap.add_argument("--latency-reps", type=int, default=100)
    ap.add_argument("--cpu-sample", type=int, default=480,
                    help="instances of the oracle's timed sample (480: the whole j30 batch)")
    ap.add_argument("--cpu-iterations", type=int, default=0, help="iterations of the oracle sample (0: the step's)")
    ap.add_argument("--reference-sample", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", choices=("seeds", "lpt"), default="seeds",
                    help="seeds: each rank its own batch (weak scaling); lpt: one batch split over the ranks "
                         "by estimated cost, results gathered on rank 0 (strong scaling)")
    ap.add_argument("--coop-blocks", type=int, default=4,
                    help="co-operating searches per instance in the cooperation measurement (0 skips it)")
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
        print(json.dumps({"serving": serving_run(R, I, 0, args.serving_family, args.serving_rate,
                                                 args.serving_seconds, args.serving_iterations,
                                                 drain_s=args.serving_drain,
                                                 slice_iterations=args.serving_slice)}), flush=True)
        return 0
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
