"""The benchmark's reference arm runs the CPU oracle (no GPU) and prints
one JSON line in the benchmark's format."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--reference-sample", "4", "--reference-iterations", "5"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "schedules/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["iterations"] == 1000 and d["config"]["workload"].startswith("mixed_batch")
    assert d["config"]["reference_sample"] == 4 and d["config"]["reference_iterations"] == 5


def test_committed_counters_match_the_kernel_source():
    """The ncu DRAM figures the bench line quotes are used only while the
    kernel source is the one captured; after a change of the kernel they
    read as null until it is captured again."""
    import pytest
    sys.path.insert(0, ROOT)
    import bench
    c = bench.load_counters()
    if c is None:
        pytest.skip("the kernel changed since its ncu capture: the bench line reports no DRAM traffic")
    assert c["dram_bytes_per_launch"] > 0
