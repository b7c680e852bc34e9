"""The native request server's book-keeping on the CPU (include/lrs.h,
lrs_server_*; a runner that sleeps stands in for the solver): admission
never exceeds the slots or the HBM budget, requests are admitted in arrival
order once they have arrived, every request completes once, a failing
request is reported without stopping the loop, and the summary's latency
percentiles match the recorded times."""
import threading
import time

import numpy as np
import pytest

import bench
from paper_2311_03824_gb300 import lrs as L
from paper_2311_03824_gb300 import serve as S


def dummy_inputs(rq):
    return np.zeros(1, np.float32), np.zeros(1, np.float32)


def overlaps_ok(res, slots, budget):
    """At every start, the requests running (including it) fit the budget,
    and their groups the slots (requests batched into one launch share a
    slot; a queue that forms, e.g. on a loaded host, makes such batches)."""
    for r in res:
        running = [o for o in res if o.start <= r.start < o.end]
        assert len({o.group for o in running}) <= slots, (r.rid, len(running))
        assert sum(o.footprint for o in running) <= budget


def test_admission_respects_slots_and_budget():
    reqs = bench.c4_requests(40, seed=9, T=10)
    bench.poisson_arrivals(reqs, rate=2000.0, seed=3)
    fps = [S.footprint_bytes(r, host_inputs=True) for r in reqs]
    budget = int(2.5 * max(fps))
    lock = threading.Lock()
    seen = []

    def run(rq, grid, worker):
        with lock:
            seen.append(rq.rid)
        time.sleep(0.002 + 0.001 * (rq.rid % 3))
        return L.LRS_OK

    srv = S.Server(budget, slots=3, runner=run)
    res = srv.run(reqs, dummy_inputs)
    assert sorted(r.rid for r in res) == list(range(40))
    assert sorted(seen) == list(range(40))
    assert all(r.error is None for r in res)
    arrival_order = [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]
    assert [r.rid for r in sorted(res, key=lambda r: r.admitted)] == arrival_order   # FIFO
    overlaps_ok(res, 3, budget)
    assert srv.peak_running <= 3
    for r in res:
        assert r.start >= r.arrival - 1e-3 and r.end >= r.start
        assert r.footprint == S.footprint_bytes(reqs[r.rid], host_inputs=True)
    summ = S.summarize(res, srv.makespan, reqs)
    lat = np.array([r.latency for r in res])
    assert summ["p50_latency_s"] == pytest.approx(np.percentile(lat, 50))
    assert summ["p99_latency_s"] == pytest.approx(np.percentile(lat, 99))
    assert summ["failed"] == 0 and summ["column_iters_per_s"] > 0


def test_failed_request_is_reported_and_loop_continues():
    reqs = bench.c4_requests(6, seed=2, T=5)

    def run(rq, grid, worker):
        return L.LRS_ERR_NUMERICAL if rq.rid == 2 else L.LRS_OK

    srv = S.Server(10 ** 15, slots=2, runner=run)
    res = srv.run(reqs, dummy_inputs)
    assert [r.rid for r in res] == list(range(6))
    assert res[2].error and "LRS_ERR_NUMERICAL" in res[2].error
    summ = S.summarize(res, srv.makespan)
    assert summ["failed"] == 1 and summ["failures"][0][0] == 2


def test_request_larger_than_budget_is_rejected():
    reqs = bench.c4_requests(3, seed=1)
    srv = S.Server(1, slots=1, runner=lambda rq, g, w: L.LRS_OK)
    res = srv.run(reqs, dummy_inputs)
    assert all(r.error and "budget" in r.error for r in res)


def test_wait_times_out_on_an_unfinished_request():
    release = threading.Event()

    def run(rq, grid, worker):
        release.wait(5.0)
        return L.LRS_OK

    srv, cb = L.lrs_server_create(10 ** 12, 1, 0, lambda req, g, w: run(None, g, w))
    rq = bench.c4_requests(1, seed=4)[0]
    y, a = dummy_inputs(rq)
    req = S.native_request(rq, y, a)
    t = L.lrs_server_submit(srv, req)
    with pytest.raises(L.LrsError) as e:
        L.lrs_server_wait(srv, t, 50)
    assert e.value.status == L.LRS_ERR_TIMEOUT
    release.set()
    res = L.lrs_server_wait(srv, t, -1)
    assert res.status == L.LRS_OK and res.grid >= 16
    L.lrs_server_destroy(srv)
    del cb


def test_mix_laws():
    reqs = bench.c4_requests(400, seed=5)
    g = [r for r in reqs if r.kind == "gaussian"]
    d = [r for r in reqs if r.kind == "dft"]
    assert 0.6 < len(g) / len(reqs) < 0.8
    assert all(256 <= r.n <= 4096 and r.n % 64 == 0 for r in g)
    assert all(64 <= r.q <= 1024 and r.q % 16 == 0 for r in reqs)
    assert all(2 <= r.r <= 10 for r in reqs)
    assert all(0.15 * r.n - 1 <= r.m <= 0.4 * r.n + 1 for r in reqs)
    assert all((r.nx, r.ny) in ((64, 64), (128, 128)) for r in d)


def test_compatible_gaussian_requests_are_admitted_together():
    """batch = 3: requests queued behind a Gaussian head with the same rank,
    A_k form and iteration count join its batch (up to 3, one slot) while the
    budget allows; any other request ends the batch; FIFO order is kept."""
    blocker = S.Request(0, "gaussian", n=4096, q=2048, r=8, m=512, rho=40, seed=1, T=100,
                        a_dtype=L.LRS_A_FP32)
    g = dict(kind="gaussian", n=256, q=64, m=80, rho=3, seed=2, T=100)
    reqs = [blocker] + [S.Request(i, r=3, **g) for i in (1, 2, 3, 4)] + \
        [S.Request(5, r=4, **g)] + [S.Request(i, r=3, **g) for i in (6, 7)] + \
        [S.Request(8, "dft", n=64 * 64, q=16, r=2, m=600, rho=20, seed=3, T=100, nx=64, ny=64)]
    budget = S.footprint_bytes(blocker, host_inputs=True)
    assert sum(S.footprint_bytes(r, host_inputs=True) for r in reqs[1:]) <= budget

    def run(rq, grid, worker):
        if rq.rid == 0:
            time.sleep(0.3)            # everything else queues behind it meanwhile
        return L.LRS_OK

    res = S.Server(budget, slots=8, runner=run, batch=3).run(reqs, dummy_inputs)
    by = {r.rid: r for r in res}
    assert [by[i].admitted for i in range(9)] == list(range(9))
    groups = {i: (by[i].group, by[i].group_size) for i in range(9)}
    assert groups == {0: (0, 1), 1: (1, 3), 2: (1, 3), 3: (1, 3), 4: (4, 1), 5: (5, 1),
                      6: (6, 2), 7: (6, 2), 8: (8, 1)}
    assert all(r.error is None for r in res)
    for i in (2, 3):                   # one worker, one start and end per batch
        assert abs(by[i].start - by[1].start) < 1e-3 and abs(by[i].end - by[1].end) < 1e-3
