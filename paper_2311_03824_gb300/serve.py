"""Serving loop: many AltGDmin-LR+S reconstruction problems solved on one GPU
with continuous batching.

Requests (Gaussian or row-masked 2D-DFT problems of any n, q, r, m, rho)
arrive over time.  A request is admitted as soon as a slot is free and its
device footprint fits the HBM budget left by the requests in flight; each
admitted request runs on its own CUDA stream through the C ABI (its A_k or
masks, U, B, S stay on the device for all of its iterations), so the work of
concurrent requests overlaps on the GPU; the persistent sweep of a Gaussian
request gets a share of the SMs (`lrs_options.grid`).  Finished requests
release their slot and memory, which admits the next ones.  Latency is
completion minus arrival, queueing and input generation included.

Every solver step runs in the library's kernels; this module only orders the
calls, generates the synthetic inputs and keeps the books.
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
    rel_err: float
    outputs: Optional[tuple] = None
    error: Optional[str] = None

    @property
    def latency(self):
        return self.end - self.arrival


def footprint_bytes(req: Request) -> int:
    """Device bytes a request holds while it runs (inputs, the stored operator,
    the exact copy kept for the refinement of low-precision forms, the task
    engine's per-column scratch, the iterate), with 10 % headroom."""
    n, q, r, m, rho = req.n, req.q, req.r, req.m, req.rho
    if req.kind == "dft":
        b = q * m * (8 + 4 + 8 + 4) + q * n * 8 + 8 * n * r * 8 + q * max(rho, 1) * 12
    else:
        ns = (n + 31) // 32 * 32
        eb = {L.LRS_A_FP32: 4, L.LRS_A_BF16: 2, L.LRS_A_FP8_HI: 1, L.LRS_A_FP8_HILO: 2}[req.a_dtype]
        gen = q * m * n * 4                        # the generated FP32 A_k (freed after set-up)
        stored = q * m * ns * eb
        exact = q * m * n * 4 if req.a_dtype != L.LRS_A_FP32 else 0
        scratch = q * (n + ns + 2 * m + 16 * 16 * 2 + 4 * 16 * m) * 4
        b = gen + stored + exact + scratch + q * m * 8
    return int(b * 1.1) + (64 << 20)


def c4_requests(count: int, seed: int = 5, T: int = 100):
    """The serving mix: 70 % Gaussian problems with BF16-stored A_k,
    n = 64 round(2^U[8,12] / 64), q = 16 round(2^U[6,10] / 16), r ~ U{2..10},
    m = round(U[0.15, 0.4] n), rho = round(U[0.01, 0.02] n); 30 % DFT problems
    on 64 x 64 or 128 x 128 frames with the same laws for q, r, rho and
    m / n in [0.15, 0.40] (64 x 64) or [0.10, 0.125] (128 x 128: one frame and
    its m samples must fit one CTA's shared memory)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        q = int(16 * round(2 ** rng.uniform(6, 10) / 16))
        r = int(rng.integers(2, 11))
        if rng.uniform() < 0.7:
            n = int(64 * round(2 ** rng.uniform(8, 12) / 64))
            m = int(round(rng.uniform(0.15, 0.4) * n))
            rho = max(1, int(round(rng.uniform(0.01, 0.02) * n)))
            out.append(Request(i, "gaussian", n, q, r, max(m, r), rho, seed * 100003 + i, T))
        else:
            side = 64 if rng.uniform() < 0.5 else 128
            n = side * side
            frac = rng.uniform(0.15, 0.4) if side == 64 else rng.uniform(0.10, 0.125)
            m = int(round(frac * n))
            rho = max(1, int(round(rng.uniform(0.01, 0.02) * n)))
            out.append(Request(i, "dft", n, q, r, m, rho, seed * 100003 + i, T, nx=side, ny=side,
                               a_dtype=L.LRS_A_FP32))
    return out


def poisson_arrivals(reqs, rate, seed=6):
    """Arrival times of a Poisson process of the given rate (requests/s)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    for rq in reqs:
        t += rng.exponential(1.0 / rate)
        rq.arrival = t
    return reqs


def solve_on_device(req: Request, stream, grid: int = 0, keep_outputs: bool = False):
    """Generate the request's synthetic inputs on its stream, solve it through
    the C ABI (lrs_init + T x GDmin iterations) and return (outputs or None,
    relative error of X = U B + S against X*)."""
    import torch
    from lrsgen import FourierInstance
    from lrsgen.device import DeviceGaussianInstance
    with torch.cuda.stream(stream):
        if req.kind == "dft":
            inst = FourierInstance(nx=req.nx, ny=req.ny, q=req.q, r=req.r, m=req.m, rho=req.rho,
                                   seed=req.seed)
            s = L.Solver(req.n, req.m, req.q, req.r, req.rho, kind=L.LRS_OP_DFT2D_MASK,
                         nx=req.nx, ny=req.ny, stream=stream)
            s.set_measurements(np.ascontiguousarray(inst.Y, np.complex64),
                               np.ascontiguousarray(inst.masks, np.int32))
            Xs = inst.Xstar
        else:
            inst = DeviceGaussianInstance(req.n, req.q, req.r, req.m, req.rho, req.seed)
            s = L.Solver(req.n, req.m, req.q, req.r, req.rho, stream=stream,
                         a_dtype=req.a_dtype, grid=grid, engine=2)
            s.set_measurements(inst.Y, inst.A)
            inst.free()
            Xs = inst.Xstar
        try:
            s.init()
            s.iterate(req.T)
            out = s.get()
        finally:
            s.close()
    U, B, Si, Sv = out
    dt = np.complex128 if req.kind == "dft" else np.float64
    X = U.astype(dt) @ B.astype(dt)
    for k in range(req.q):
        X[Si[k], k] += Sv[k]
    err = float(np.linalg.norm(X - Xs) / np.linalg.norm(Xs))
    return (out if keep_outputs else None), err


class Server:
    """Continuous-batching request loop (see the module docstring).

    run_request(req, slot_info) -> (outputs, rel_err) does the work of one
    request; the default solves it on the GPU.  `slots` requests run at once
    at most, and the footprints of the requests in flight never exceed
    `hbm_budget` bytes."""

    def __init__(self, hbm_budget: int, slots: int = 8, sms: int = 152,
                 run_request: Optional[Callable] = None, keep_outputs: bool = False):
        self.budget = int(hbm_budget)
        self.slots = int(slots)
        self.sms = int(sms)
        self.keep_outputs = keep_outputs
        self._run = run_request
        self._lock = threading.Condition()
        self.in_use = 0
        self.running = 0
        self.peak_in_use = 0
        self.peak_running = 0
        self.makespan = 0.0

    def grid_for(self, running_after: int) -> int:
        """CTAs of a Gaussian request's persistent sweep: the GPU's two CTAs per
        SM shared by the requests that will be running."""
        return max(16, (2 * self.sms) // max(1, running_after))

    def run(self, reqs, start_clock: Optional[float] = None):
        """Serve `reqs` (admitted in arrival order); returns the Results in rid
        order."""
        import queue
        reqs = sorted(reqs, key=lambda r: r.arrival)
        for rq in reqs:
            if footprint_bytes(rq) > self.budget:
                raise ValueError(f"request {rq.rid} needs more than the whole HBM budget")
        pending = list(reqs)
        results = {}
        t0 = time.perf_counter() if start_clock is None else start_clock
        work = queue.Queue()
        streams = []
        if self._run is None:
            import torch
            streams = [torch.cuda.Stream() for _ in range(self.slots)]

        def worker(wi):
            while True:
                item = work.get()
                if item is None:
                    return
                rq, grid, start = item
                outs, err, msg = None, math.inf, None
                try:
                    if self._run is not None:
                        outs, err = self._run(rq, dict(grid=grid, worker=wi))
                    else:
                        outs, err = solve_on_device(rq, streams[wi], grid, self.keep_outputs)
                except Exception as ex:  # the request fails; the loop goes on
                    msg = f"{type(ex).__name__}: {ex}"
                finally:
                    end = time.perf_counter() - t0
                    with self._lock:
                        self.in_use -= footprint_bytes(rq)
                        self.running -= 1
                        self._lock.notify_all()
                results[rq.rid] = Result(rq.rid, rq.kind, rq.arrival, start, end, err, outs, msg)

        threads = [threading.Thread(target=worker, args=(i,), daemon=True)
                   for i in range(self.slots)]
        for th in threads:
            th.start()
        # admission: FIFO by arrival; a request waits until it has arrived, a
        # slot is free and its footprint fits
        while pending:
            rq = pending[0]
            now = time.perf_counter() - t0
            if rq.arrival > now:
                time.sleep(min(rq.arrival - now, 0.01))
                continue
            fp = footprint_bytes(rq)
            with self._lock:
                while not (self.running < self.slots and self.in_use + fp <= self.budget):
                    self._lock.wait(0.01)
                self.in_use += fp
                self.running += 1
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                self.peak_running = max(self.peak_running, self.running)
                grid = self.grid_for(self.running)
            pending.pop(0)
            work.put((rq, grid, time.perf_counter() - t0))
        for _ in threads:
            work.put(None)
        for th in threads:
            th.join()
        self.makespan = time.perf_counter() - t0
        return [results[k] for k in sorted(results)]


def summarize(results, makespan, reqs=None):
    """Latency percentiles, throughput (requests/s and column-iterations/s),
    the errors reached, and the failed and unsolved requests."""
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency for r in ok])
    out = dict(requests=len(results), failed=len(results) - len(ok), makespan_s=makespan,
               throughput_req_s=len(ok) / makespan if makespan > 0 else math.inf,
               p50_latency_s=float(np.percentile(lat, 50)) if len(lat) else None,
               p99_latency_s=float(np.percentile(lat, 99)) if len(lat) else None,
               mean_latency_s=float(lat.mean()) if len(lat) else None,
               max_rel_err=float(max(r.rel_err for r in ok)) if ok else None)
    errs = np.array([r.rel_err for r in ok])
    if len(errs):
        out["rel_err_p50"] = float(np.median(errs))
        out["solved_1e-3"] = int(np.sum(errs <= 1e-3))
    out["failures"] = [(r.rid, r.error[:160]) for r in results if r.error is not None][:6]
    if reqs is not None:
        by = {rq.rid: rq for rq in reqs}
        ci = sum(by[r.rid].q * by[r.rid].T for r in ok)
        out["column_iters_per_s"] = ci / makespan if makespan > 0 else math.inf
        out["unsolved"] = [(r.rid, by[r.rid].kind, by[r.rid].n, by[r.rid].q, by[r.rid].r,
                            by[r.rid].m, by[r.rid].rho, round(r.rel_err, 4))
                           for r in ok if r.rel_err > 1e-3][:8]
    return out
