"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (the task engine, every column in flight, the task shape chosen by the
autotuner on the first iteration for the Gaussian cases).

* n=1000, q=1000, r=5, m=150, rho=10 (float32 A_k): from the GPU's own
  iterates t = 0 (after lrs_init), 20 and 60, one GDmin iteration on the GPU
  against one FP64 oracle iteration from the same state;
* n=4096, q=2048, r=10, m=512, rho=40 (A_k drawn on the device, 17 GB): the
  whole problem is beyond the oracle, so the per-column outputs b_k and s_k
  of one GPU iteration are checked on sampled columns, whose A_k are copied
  back and given to the oracle with the GPU's U, B, S;
* 128 x 128 DFT frames, q=256, r=6, m=2048, rho=82: one-step parity from the
  GPU's iterates t = 0 and 30.

Bars as in the other parity tests (tests/gpu_helpers.py): b_k and s_k of a
column depend only on that column and on U_t, so they are compared on every
decidable column (supports identical, values within 1e-5), decided by the
probed oracle step (FP64 margin above 1e-6 and above ten times its float32
change, same float32 support).  U_{t+1} mixes all columns through the
gradient, so the whole X is compared (1e-5) at steps where every column is
decidable; the full-problem cases must have such steps.
"""
import numpy as np
import pytest

import oracle.altgdmin_lrs as O
from lrsgen import C1, C2, C3, FourierInstance, GaussianInstance
from tests.gpu_helpers import (Problem, check_records, compare_step, gpu_available,
                               new_fourier_solver, new_solver, probe_step, state_from_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


@pytest.mark.parametrize("opts", [dict(autotune=1), dict(engine=3)],
                         ids=["default", "resident"])
def test_one_step_gaussian_n1000_q1000(opts):
    cfg = {k: v for k, v in C1.items() if k != "T"}
    inst = GaussianInstance(**cfg)
    P = Problem.gaussian(inst)
    s = new_solver(inst, **opts)
    s.init()
    t, recs = 0, []
    try:
        for target in (0, 20, 60):
            s.iterate(target - t)
            t = target
            g = s.get()
            eta, _ = s.progress()
            st64, _, dec, dev = probe_step(P, state_from_gpu(g, inst.n, t, eta, np.float64))
            s.iterate(1)
            t += 1
            recs.append(compare_step(st64, dec, s.get(), dev=dev))
    finally:
        s.close()
    check_records(recs, min_whole=1)


def test_sampled_columns_gaussian_n4096_q2048():
    import torch
    from paper_2311_03824_gb300 import Solver
    from lrsgen.device import DeviceGaussianInstance
    cfg = {k: v for k, v in C2.items() if k != "T"}
    dev = DeviceGaussianInstance(**cfg)
    stream = torch.cuda.Stream()
    n, q, r, m, rho = cfg["n"], cfg["q"], cfg["r"], cfg["m"], cfg["rho"]
    s = Solver(n, m, q, r, rho, stream=stream, autotune=1)
    try:
        s.set_measurements(dev.Y, dev.A)
        s.init()
        s.iterate(5)
        U, B, Si, Sv = s.get()                 # iterate t = 5
        eta, _ = s.progress()
        s.iterate(1)
        U1, B1, S1i, S1v = s.get()             # b_k, s_k of iteration 6 (computed with U_5)
    finally:
        s.close()
    ks = np.sort(np.random.default_rng(17).choice(q, 8, replace=False))
    kt = torch.as_tensor(ks, device=dev.A.device)
    A = dev.A[kt].cpu().numpy()
    Y = dev.Y[kt].cpu().numpy()
    dev.free()
    P = Problem(O.GaussianOperator(A), O.GaussianOperator(A, np.float32), Y, r, rho)
    st64, _, dec, dev = probe_step(P, state_from_gpu((U, B[:, ks], Si[ks], Sv[ks]), n, 5, eta,
                                                     np.float64))
    rec = compare_step(st64, dec, (U1, B1[:, ks], S1i[ks], S1v[ks]), whole=False, dev=dev)
    check_records([rec], min_whole=0, max_excluded=0.25)


def test_one_step_fourier_128x128():
    cfg = {k: v for k, v in C3.items() if k != "T"}
    inst = FourierInstance(**cfg)
    P = Problem.fourier(inst)
    s = new_fourier_solver(inst)
    s.init()
    t, recs = 0, []
    try:
        for target in (0, 30):
            s.iterate(target - t)
            t = target
            g = s.get()
            eta, _ = s.progress()
            st64, _, dec, dev = probe_step(P, state_from_gpu(g, inst.n, t, eta, np.complex128))
            s.iterate(1)
            t += 1
            recs.append(compare_step(st64, dec, s.get(), dev=dev))
    finally:
        s.close()
    check_records(recs, min_whole=0, max_excluded=0.05)
