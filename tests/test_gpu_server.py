"""GPU tests of the continuous-batching server (rcpsp_server_*)."""
import os
import time

import numpy as np
import pytest

from paper_1711_04556_gb300 import instances as I
from paper_1711_04556_gb300 import rcpsp as R

pytestmark = pytest.mark.gpu
NPROC = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_04556_gb300 import build as B
    B.build()


def drain(srv, want, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < want and time.time() - t0 < timeout:
        for c in srv.poll(wait_ms=50):
            got[c["tag"]] = c
    assert len(got) == want, f"{len(got)} of {want} requests finished"
    return got


def same(a, b):
    for k in ("status", "best_cmax", "iterations", "evaluated", "work", "mode", "cp"):
        assert a[k] == b[k], k
    assert a["best_W"].tolist() == b["best_W"].tolist()
    assert a["best_S"].tolist() == b["best_S"].tolist()


def test_result_is_the_same_alone_and_in_the_mix(oracle):
    x = I.generate(7, 30, 4, 180, 50, stream=21)
    with R.Server(0, slots=4, max_batch=32) as srv:
        srv.submit(x, tag=0, iterations=200, delta=20, tabu_len=60)
        alone = drain(srv, 1)[0]
        mix = I.config_batch("j30_batch", 120, first=50) + I.config_batch("j120_batch", 6)
        rng = np.random.default_rng(1)
        order = rng.permutation(len(mix))
        for k, j in enumerate(order):
            srv.submit(mix[j], tag=1 + int(j), iterations=200, delta=20, tabu_len=60)
            if k == len(order) // 2:
                srv.submit(x, tag=999, iterations=200, delta=20, tabu_len=60)
        got = drain(srv, len(mix) + 1)
        st = srv.stats()
    same(alone, got[999])
    ref = oracle.tabu_search(x, 200, 20, 60, 0, 1)
    assert alone["best_cmax"] == ref["best_cmax"] and alone["evaluated"] == ref["evaluated"]
    assert alone["best_W"].tolist() == ref["best_W"].tolist()
    refs = oracle.tabu_search_batch(mix[:24], [(200, 20, 60, 0, 1)] * 24, NPROC)
    for j in range(24):
        assert got[1 + j]["best_cmax"] == refs[j]["best_cmax"]
        assert got[1 + j]["evaluated"] == refs[j]["evaluated"]
    assert st["completed"] == len(mix) + 2 and st["batches"] >= 4
    # batches overlapped: some batch started before an earlier one had finished
    spans = sorted({(c["t_launch_ns"], c["t_done_ns"]) for c in got.values()})
    assert any(b[0] < a[1] for a, b in zip(spans, spans[1:]))


def test_admission_respects_the_memory_budget():
    insts = I.config_batch("j30_batch", 60, first=400)
    budget = 64 * 1024
    with R.Server(0, slots=4, max_batch=64, memory_budget=budget) as srv:
        for k, x in enumerate(insts):
            srv.submit(x, tag=k, iterations=50, delta=20, tabu_len=60)
        got = drain(srv, len(insts))
        st = srv.stats()
    assert all(c["status"] == 0 for c in got.values())
    assert st["max_inflight_bytes"] <= budget and st["batches"] > 1


def test_invalid_request_is_rejected():
    x = I.generate(3, 10, 2, 150, 50, stream=22)
    req = x.req.copy()
    req[x.m] = x.cap[0] + 1
    bad = I.Instance(x.n, x.m, x.dur, x.cap, req, x.succ_off, x.succ)
    with R.Server(0) as srv:
        with pytest.raises(R.RcpspError) as e:
            srv.submit(bad, tag=1)
        assert e.value.code == -4
        assert srv.stats()["rejected"] == 1


def test_time_slicing_gives_uninterrupted_results(oracle):
    """With slice_iterations the server runs long requests in slices (state
    kept between batches, requests requeued); every result is still the
    uninterrupted search's, and short requests submitted later finish first."""
    longs = I.config_batch("j30_batch", 40, first=150) + I.config_batch("j120_batch", 3, first=40)
    shorts = I.config_batch("j30_batch", 8, first=400)
    with R.Server(0, slots=4, max_batch=16, slice_iterations=30) as srv:
        for k, x in enumerate(longs):
            srv.submit(x, tag=k, iterations=150, delta=0, tabu_len=0, stop_at_cp=False)
        for k, x in enumerate(shorts):
            srv.submit(x, tag=1000 + k, iterations=20, delta=0, tabu_len=0, stop_at_cp=False)
        got = drain(srv, len(longs) + len(shorts))
        st = srv.stats()
    assert st["requeued"] > 0
    params = [(150,) + I.search_params(x.n - 2) + (0, 0) for x in longs]
    refs = oracle.tabu_search_batch(longs, params, NPROC)
    for k, r in enumerate(refs):
        g = got[k]
        assert g["status"] == 0 and g["iterations"] == 150
        assert g["best_cmax"] == r["best_cmax"] and g["evaluated"] == r["evaluated"] and g["work"] == r["work"]
        assert g["best_W"].tolist() == r["best_W"].tolist()
    last_short = max(got[1000 + k]["t_done_ns"] for k in range(len(shorts)))
    last_long = max(got[k]["t_done_ns"] for k in range(len(longs)))
    assert last_short < last_long
