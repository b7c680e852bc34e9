"""The serving loop's book-keeping on the CPU (a fake solver that sleeps):
admission never exceeds the slots or the HBM budget, requests start in
arrival order once they have arrived, every request completes once, a
failing request is reported without stopping the loop, and the summary's
latency percentiles match the recorded times."""
import threading
import time

import numpy as np
import pytest

from paper_2311_03824_gb300 import serve as S


def test_admission_respects_slots_and_budget():
    reqs = S.c4_requests(40, seed=9, T=10)
    S.poisson_arrivals(reqs, rate=2000.0, seed=3)
    budget = int(2.5 * max(S.footprint_bytes(r) for r in reqs))
    log, lock = [], threading.Lock()
    srv = S.Server(budget, slots=3)

    def run(rq, info):
        with lock:
            log.append(rq.rid)
            assert srv.running <= 3 and srv.in_use <= budget
        time.sleep(0.002 + 0.001 * (rq.rid % 3))
        return None, 1e-7

    srv._run = run
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == list(range(40))
    assert srv.peak_running <= 3 and srv.peak_in_use <= budget
    assert all(r.error is None for r in res)
    assert log == [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]   # FIFO
    for r in res:
        assert r.start >= r.arrival - 1e-6 and r.end >= r.start
    summ = S.summarize(res, srv.makespan, reqs)
    lat = np.array([r.latency for r in res])
    assert summ["p50_latency_s"] == pytest.approx(np.percentile(lat, 50))
    assert summ["p99_latency_s"] == pytest.approx(np.percentile(lat, 99))
    assert summ["failed"] == 0 and summ["column_iters_per_s"] > 0


def test_failed_request_is_reported_and_loop_continues():
    reqs = S.c4_requests(6, seed=2, T=5)

    def run(rq, info):
        if rq.rid == 2:
            raise RuntimeError("boom")
        return None, 0.0

    srv = S.Server(10 ** 15, slots=2, run_request=run)
    res = srv.run(reqs)
    assert [r.rid for r in res] == list(range(6))
    assert res[2].error and "boom" in res[2].error
    summ = S.summarize(res, srv.makespan)
    assert summ["failed"] == 1 and summ["failures"][0][0] == 2


def test_request_larger_than_budget_is_rejected():
    reqs = S.c4_requests(3, seed=1)
    with pytest.raises(ValueError):
        S.Server(1, slots=1, run_request=lambda rq, i: (None, 0.0)).run(reqs)


def test_mix_laws():
    reqs = S.c4_requests(400, seed=5)
    g = [r for r in reqs if r.kind == "gaussian"]
    d = [r for r in reqs if r.kind == "dft"]
    assert 0.6 < len(g) / len(reqs) < 0.8
    assert all(256 <= r.n <= 4096 and r.n % 64 == 0 for r in g)
    assert all(64 <= r.q <= 1024 and r.q % 16 == 0 for r in reqs)
    assert all(2 <= r.r <= 10 for r in reqs)
    assert all(0.15 * r.n - 1 <= r.m <= 0.4 * r.n + 1 for r in g)
    assert all((r.nx, r.ny) in ((64, 64), (128, 128)) and r.m <= 2048 for r in d)
