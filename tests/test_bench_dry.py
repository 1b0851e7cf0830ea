"""bench.py's own arm, run end to end on the CPU against a stand-in solver.

The stand-in replaces the CUDA library and torch's CUDA objects in a child
process, so the benchmark's control flow -- warm-up, timed steps, end to
end steps, the per-instance and latency samples, the roofline and counters,
both ways of splitting instances -- runs and prints its JSON line without a
GPU.  It checks the line's shape, not its numbers (the GPU runs measure).
"""
import contextlib
import json
import os
import subprocess
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(argv):
    import numpy as np
    import torch

    class Event:
        def __init__(self, **_):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 40.0

    torch.cuda.is_available = lambda: True
    torch.cuda.set_device = lambda *_: None
    torch.cuda.Stream = lambda *a, **k: object()
    torch.cuda.Event = Event
    torch.cuda.synchronize = lambda *_: None
    torch.cuda.stream = lambda st: contextlib.nullcontext()
    torch.cuda.get_device_properties = lambda d: types.SimpleNamespace(multi_processor_count=152)
    torch.cuda.get_device_name = lambda d: "stand-in GPU"
    empty = torch.empty
    torch.empty = lambda *a, **k: empty(16, dtype=k.get("dtype"))
    sys.path.insert(0, ROOT)
    from paper_1711_04556_gb300 import build as B
    from paper_1711_04556_gb300 import rcpsp as R
    B.build = lambda *a, **k: None
    R.measure_peaks = lambda d: {"int32_ops_per_s": 20e12, "smem_bytes_per_s": 40e12, "int32_ops_per_clk_sm": 64.0,
                                 "smem_bytes_per_clk_sm": 128.0, "sm_clock_mhz": 2070.0, "sms": 152}

    class Solver:
        def __init__(self, device):
            self.insts, self.next, self.launches = {}, 0, 0

        def load(self, insts):
            ids = list(range(self.next, self.next + len(insts)))
            self.insts.update(zip(ids, insts))
            self.next += len(insts)
            return ids

        def autotune(self, ids, **_):
            return (4, 12, 1)

        def search(self, ids, **_):
            self.launches += 1

        def results(self, ids):
            return [dict(best_cmax=40, cp=35, evaluated=1000, work=5000, iterations=1000, mode=1 + i % 2, status=0,
                         t_start_ns=0, t_end_ns=20_000_000, best_W=np.arange(self.insts[i].n),
                         best_S=np.zeros(self.insts[i].n), placements=1000 * self.insts[i].n, steps_done=5000,
                         update_units=100_000, succ_pushes=50_000, kept_words=0) for i in ids]

        def last_launches(self):
            return [dict(searches=4, group_size=4, warps=12, cluster_size=1, ctas=4, prefix_reuse=0,
                         shape_source=0, slices=1, smem_bytes=1 << 16)]

        def kernel_launches(self):
            return self.launches

        def transfer_bytes(self):
            return self.launches * 1000, self.launches * 100

        def free(self, ids):
            pass

        def close(self):
            pass

    R.Solver = Solver
    import bench

    class Sampler:
        def __init__(self, *_):
            pass

        def stop(self):
            return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 1}

    bench.ClockSampler = Sampler
    sys.argv = ["bench.py"] + argv
    bench.main()


def run(*extra):
    base = ["--steps", "3", "--warmup", "3", "--serving-seconds", "0", "--coop-blocks", "0", "--latency-reps", "2",
            "--plain-sample", "2", "--no-cpu-baseline", "--j120-steps", "1", "--j30-steps", "2"]
    r = subprocess.run([sys.executable, os.path.abspath(__file__)] + base + list(extra), capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_default_line_has_every_key():
    d = run()
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "cpu_baseline", "clocks"):
        assert k in d, k
    assert d["scaling"] == "weak" and d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["gpu_launches"] == 3 and d["config"]["workload"].startswith("mixed_batch")
    assert d["config"]["shapes_from"].startswith("rcpsp_autotune")
    assert d["config"]["instances"] == 1024 and d["quality"]["instances"] == 1024
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "smem", "kept_state", "peak_basis"):
        assert k in d["roofline"], k
    assert "measured" in d["roofline"]["peak_basis"]
    # the fraction follows from the printed counters and the measured peak
    r = d["roofline"]
    assert abs(r["achieved"] - r["ops_per_launch"] / (d["ms_per_step"] / 1000) / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12 and 0 < r["frac"] < 1
    assert 0 < r["smem"]["frac"] < 1
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert set(d["configs"]) == {"j30_batch", "j120_batch"}
    j30 = d["configs"]["j30_batch"]
    assert j30["config"]["instances"] == 480 and j30["value"] > 0 and "plain_per_instance_launch" in j30
    assert d["configs"]["j120_batch"]["config"]["instances"] == 600


def test_lpt_split_line():
    d = run("--shard", "lpt", "--workload", "mixed_batch")
    assert d["scaling"] == "strong" and d["quality"]["instances"] == 1024
    assert d["roofline"]["traffic"] is None


if __name__ == "__main__":
    _child(sys.argv[1:])
