"""Serving: many AltGDmin-LR+S reconstruction problems on one GPU with
continuous batching, through the library's native request server
(include/lrs.h, lrs_server_*).

The admission (first come, first served, as soon as a slot is free and the
request's device footprint fits the HBM budget left by the requests in
flight), the worker threads with one CUDA stream each, and the SM share of a
Gaussian request's persistent sweep all live in the library.  This module
only hands requests over at their arrival times, with the inputs a caller's
function produces for them, and collects the outcomes: latency is completion
minus arrival, the production of the inputs included.
"""
from __future__ import annotations

import dataclasses
import math
import threading
import time
from typing import Callable, Optional

import numpy as np

from . import lrs as L


@dataclasses.dataclass
class Request:
    rid: int
    kind: str               # "gaussian" or "dft"
    n: int
    q: int
    r: int
    m: int
    rho: int
    seed: int
    T: int = 100
    nx: int = 0
    ny: int = 0
    a_dtype: int = L.LRS_A_BF16
    arrival: float = 0.0    # seconds after the start of the run


@dataclasses.dataclass
class Result:
    rid: int
    kind: str
    arrival: float
    start: float
    end: float
    rel_err: float = math.nan
    outputs: Optional[tuple] = None
    error: Optional[str] = None
    footprint: int = 0
    grid: int = 0
    admitted: int = -1
    group: int = -1          # admission index of the first request of its batch
    group_size: int = 1

    @property
    def latency(self):
        return self.end - self.arrival


def native_request(rq: Request, y=None, A_or_mask=None, outs=None) -> L.lrs_request:
    """The lrs_request of a request (buffers: numpy host arrays or torch CUDA
    tensors, all of one kind)."""
    o = L.make_options(T=rq.T, a_dtype=rq.a_dtype if rq.kind == "gaussian" else 0,
                       nx=rq.nx, ny=rq.ny)
    req = L.lrs_request()
    req.n, req.m, req.q, req.r, req.rho = rq.n, rq.m, rq.q, rq.r, rq.rho
    req.kind = L.LRS_OP_DFT2D_MASK if rq.kind == "dft" else L.LRS_OP_GAUSSIAN
    req.opt = o
    if y is not None:
        (py, mk), (pa, _) = L._ptr(y), L._ptr(A_or_mask)
        req.y, req.A_or_mask, req.mem_kind = py, pa, mk
    if outs is not None:
        U, B, Si, Sv = outs
        req.U, req.B = L._ptr(U)[0], L._ptr(B)[0]
        req.S_idx = L._ptr(Si)[0] if rq.rho else None
        req.S_val = L._ptr(Sv)[0] if rq.rho else None
        req.out_mem_kind = 0
    req.user = rq.rid + 1          # nonzero: a null user pointer reads back as None
    return req


def footprint_bytes(rq: Request, host_inputs: bool = False) -> int:
    """Device bytes the server reserves for the request while it runs
    (lrs_request_footprint)."""
    req = native_request(rq)
    req.mem_kind = 0 if host_inputs else 1
    return L.lrs_request_footprint(req)


class Server:
    """A native request server fed at the requests' arrival times.

    make_inputs(req) -> (Y, A_or_mask) produces a request's inputs when it
    arrives (host arrays, or device tensors whose producing work is complete);
    they are kept alive until the request has finished.  runner: None (the
    library's solver) or a callable (request, grid, worker) -> lrs status
    that the server calls in its place (tests of the admission logic).
    batch: up to this many compatible Gaussian requests admitted together
    share one persistent launch per sweep (lrs_server_options.batch)."""

    def __init__(self, hbm_budget: int, slots: int = 8, sms: int = 0,
                 runner: Optional[Callable] = None, keep_outputs: bool = False, batch: int = 0):
        self.budget = int(hbm_budget)
        self.slots = int(slots)
        self.sms = int(sms)
        self.batch = int(batch)
        self.keep_outputs = keep_outputs
        self._runner = runner
        self.makespan = 0.0
        self.peak_running = 0

    def run(self, reqs, make_inputs: Callable, start_clock: Optional[float] = None):
        """Serve `reqs` (handed over in arrival order); returns the Results in
        rid order."""
        by_rid = {rq.rid: rq for rq in reqs}
        runner = None
        if self._runner is not None:
            runner = lambda req, grid, worker: self._runner(by_rid[req.user - 1], grid, worker)
        srv, cb = L.lrs_server_create(self.budget, self.slots, self.sms, runner, self.batch)
        t0 = time.perf_counter() if start_clock is None else start_clock
        order = sorted(reqs, key=lambda r: r.arrival)
        tickets, held, submitted = {}, {}, {}
        failures = {}

        def submitter():
            for rq in order:
                now = time.perf_counter() - t0
                if rq.arrival > now:
                    time.sleep(rq.arrival - now)
                try:
                    y, a = make_inputs(rq)
                    outs = None
                    if self.keep_outputs:
                        dt = np.complex64 if rq.kind == "dft" else np.float32
                        outs = (np.empty((rq.r, rq.n), dt), np.empty((rq.q, rq.r), dt),
                                np.empty((rq.q, max(rq.rho, 1)), np.int32),
                                np.empty((rq.q, max(rq.rho, 1)), dt))
                    req = native_request(rq, y, a, outs)
                    held[rq.rid] = (y, a, outs, req)
                    submitted[rq.rid] = time.perf_counter() - t0
                    tickets[rq.rid] = L.lrs_server_submit(srv, req)
                except Exception as ex:   # the request fails; the loop goes on
                    failures[rq.rid] = f"{type(ex).__name__}: {ex}"

        th = threading.Thread(target=submitter, daemon=True)
        th.start()
        results = {}
        native = {}
        pending = [rq.rid for rq in order]
        while pending:
            rid = pending[0]
            if rid in failures:
                rq = by_rid[rid]
                now = time.perf_counter() - t0
                results[rid] = Result(rid, rq.kind, rq.arrival, now, now, error=failures[rid])
                pending.pop(0)
                continue
            if rid not in tickets:
                time.sleep(0.0005)
                continue
            res = L.lrs_server_wait(srv, tickets[rid], -1)
            rq = by_rid[rid]
            native[rid] = (res.submit_s, res.start_s, res.end_s)
            r = Result(rid, rq.kind, rq.arrival, res.start_s, res.end_s,
                       footprint=int(res.footprint), grid=int(res.grid),
                       admitted=int(res.admitted), group=int(res.group),
                       group_size=int(res.group_size))
            if res.status != L.LRS_OK:
                r.error = f"{L.STATUS_NAMES[res.status]}: {res.message.decode()}"
            elif self.keep_outputs:
                U, B, Si, Sv = held[rid][2]
                r.outputs = (U.T.copy(), B.T.copy(), Si[:, :rq.rho], Sv[:, :rq.rho])
            held.pop(rid, None)
            results[rid] = r
            pending.pop(0)
        th.join()
        # native times are seconds since the server's creation: one offset
        # places them all on this clock (the largest of submission time minus
        # native submission time, the closest to the clocks' true offset), so
        # that their order is the server's own
        if native:
            base = max(submitted[rid] - ns for rid, (ns, _, _) in native.items())
            for rid, (_, st, en) in native.items():
                results[rid].start = base + st
                results[rid].end = base + en
        L.lrs_server_destroy(srv)
        del cb
        self.makespan = time.perf_counter() - t0
        self.peak_running = peak_concurrency(list(results.values()))
        return [results[k] for k in sorted(results)]


def peak_concurrency(results):
    """Largest number of requests running at once (from their start and end)."""
    ev = sorted([(r.start, 1) for r in results if r.error is None] +
                [(r.end, -1) for r in results if r.error is None], key=lambda e: (e[0], e[1]))
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    return peak


def summarize(results, makespan, reqs=None):
    """Latency percentiles, throughput (requests/s and column-iterations/s),
    the errors reached, and the failed and unsolved requests."""
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency for r in ok])
    out = dict(requests=len(results), failed=len(results) - len(ok), makespan_s=makespan,
               throughput_req_s=len(ok) / makespan if makespan > 0 else math.inf,
               p50_latency_s=float(np.percentile(lat, 50)) if len(lat) else None,
               p99_latency_s=float(np.percentile(lat, 99)) if len(lat) else None,
               mean_latency_s=float(lat.mean()) if len(lat) else None)
    errs = np.array([r.rel_err for r in ok if not math.isnan(r.rel_err)])
    if len(errs):
        out["max_rel_err"] = float(errs.max())
        out["rel_err_p50"] = float(np.median(errs))
        out["solved_1e-3"] = int(np.sum(errs <= 1e-3))
    out["failures"] = [(r.rid, r.error[:160]) for r in results if r.error is not None][:6]
    if reqs is not None:
        by = {rq.rid: rq for rq in reqs}
        ci = sum(by[r.rid].q * by[r.rid].T for r in ok)
        out["column_iters_per_s"] = ci / makespan if makespan > 0 else math.inf
    return out
