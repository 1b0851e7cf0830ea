"""Timing study behind the evaluator selection rule (Sec. 5.4).

Sec. 5.4 learns which resource evaluation is faster from measured run times
of both algorithms on generated instances, because the answer depends on the
hardware.  This tool does the same on the GPU it runs on: it searches every
instance of a synthetic grid (sizes 30-300, durations up to 10/25/50,
resource strength 0.1-1.0, 4 or 8 resources) under both evaluators, reads
each search's device time per iteration from the kernel's timestamps, and
scores threshold rules of the form "capacity-indexed iff CP > K * avgCap"
(critical path and average capacity: attributes of Table 3).

    python -m paper_1711_04556_gb300.selection_study [iterations]

prints one line per K: total time if the rule picks, and how often it picks
the faster evaluator.
"""
from __future__ import annotations

import sys

import numpy as np


def grid():
    from . import instances as I
    out, seed = [], 0
    for n in (30, 60, 120, 300):
        for dmax in (10, 25, 50):
            for rs in (10, 20, 50, 70, 100):
                for m in (4, 8):
                    for _ in range(2):
                        out.append(I.generate(seed, n, m, (150, 180, 210)[seed % 3], rs, dmax=dmax, stream=77))
                        seed += 1
    return out


def measure(iterations: int = 10, device: int = 0):
    import torch
    from . import rcpsp as R
    insts = grid()
    s = R.Solver(device)
    st = torch.cuda.Stream()
    rows = []
    for n in sorted({x.n for x in insts}):
        sub = [x for x in insts if x.n == n]
        ids = s.load(sub)
        per_mode = {}
        for mode in (R.EVAL_TIME, R.EVAL_CAPACITY):
            s.autotune(ids, iterations=iterations, mode=mode, trial_iterations=2, stream=st)
            s.search(ids, iterations=iterations, mode=mode, stream=st)
            per_mode[mode] = s.results(ids)
        for x, a, b in zip(sub, per_mode[R.EVAL_TIME], per_mode[R.EVAL_CAPACITY]):
            rows.append(dict(n=x.n, m=x.m, sumR=int(x.cap.sum()), cp=R.prepare(x)["cp"],
                             t_time=(a["t_end_ns"] - a["t_start_ns"]) / max(1, a["iterations"]),
                             t_cap=(b["t_end_ns"] - b["t_start_ns"]) / max(1, b["iterations"])))
        s.free(ids)
    s.close()
    return rows


def score(rows, ks=(8, 12, 16, 20, 24, 28, 32, 40, 64)):
    cp = np.array([r["cp"] for r in rows], float)
    m = np.array([r["m"] for r in rows], float)
    sr = np.array([r["sumR"] for r in rows], float)
    tt = np.array([r["t_time"] for r in rows])
    tc = np.array([r["t_cap"] for r in rows])
    out = [("always time-indexed", tt.sum() / 1e6, float(np.mean(tt <= tc))),
           ("always capacity-indexed", tc.sum() / 1e6, float(np.mean(tc < tt))),
           ("faster of the two", np.minimum(tt, tc).sum() / 1e6, 1.0)]
    for k in ks:
        cap = cp * m > k * sr
        out.append((f"K={k}", np.where(cap, tc, tt).sum() / 1e6, float(np.mean(cap == (tc < tt)))))
    return out


if __name__ == "__main__":
    it = int(sys.argv[1]) if len(sys.argv) > 1 else 10
    for name, total_ms, acc in score(measure(it)):
        print(f"{name:26s} total {total_ms:9.1f} ms  picks the faster evaluator {100 * acc:5.1f} %")
