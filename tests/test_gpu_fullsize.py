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

Bars as in the other parity tests.  b_k and s_k of a column depend only on
that column and on U_t, so they are compared on every decidable column
(oracle margin > 1e-4): supports identical, values within 1e-5.  U_{t+1}
mixes all columns through the gradient, so the whole X is compared (1e-5)
only at steps where every column is decidable; the Gaussian cases must have
at least one such step.
"""
import numpy as np
import pytest

import oracle.altgdmin_lrs as O
from lrsgen import C1, C2, C3, FourierInstance, GaussianInstance
from tests.gpu_helpers import MARGIN_FP32, TOL, gpu_available, new_solver, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


def sorted_support(S_idx, S_val):
    o = np.argsort(S_idx, axis=1)
    return np.take_along_axis(S_idx, o, 1).astype(np.int64), np.take_along_axis(S_val, o, 1)


def state_from(U, B, S_idx, S_val, n, t, eta, dt):
    """OracleState (FP64 / complex128) of a GPU iterate (U n x r, B r x q,
    S q x rho)."""
    q = B.shape[1]
    Si, Sv = sorted_support(S_idx, S_val)
    S = np.zeros((q, n), dt)
    np.put_along_axis(S, Si, Sv.astype(dt), axis=1)
    return O.OracleState(U=U.astype(dt), B=B.astype(dt), S=S, S_idx=Si,
                         eta=eta if t else None, t=t)


def x_from(U, B, S_idx, S_val, dt):
    X = U.astype(dt) @ B.astype(dt)
    for k in range(B.shape[1]):
        X[S_idx[k], k] += S_val[k]
    return X


def check_columns(st, mg, B1, S1i, S1v, min_dec):
    """b_k and s_k of the GPU step against the oracle's on decidable columns."""
    dec = mg > MARGIN_FP32
    assert dec.sum() >= min_dec, dec.sum()
    Si, Sv = sorted_support(S1i, S1v)
    assert np.all(Si[dec] == st.S_idx[dec])
    assert rel(B1[:, dec], st.B[:, dec]) <= TOL
    So = np.take_along_axis(st.S[dec], st.S_idx[dec], 1)
    assert rel(Sv[dec], So) <= TOL
    return dec


def test_one_step_gaussian_n1000_q1000():
    cfg = {k: v for k, v in C1.items() if k != "T"}
    inst = GaussianInstance(**cfg)
    op = O.GaussianOperator(inst.A)
    s = new_solver(inst, autotune=1)
    s.init()
    t, whole = 0, 0
    try:
        for target in (0, 20, 60):
            s.iterate(target - t)
            t = target
            U, B, Si, Sv = s.get()
            eta, _ = s.progress()
            st = state_from(U, B, Si, Sv, inst.n, t, eta, np.float64)
            mg, _ = O.iterate_alg1(op, inst.Y, st, inst.rho, chunk=250)
            s.iterate(1)
            t += 1
            U1, B1, S1i, S1v = s.get()
            dec = check_columns(st, mg, B1, S1i, S1v, min_dec=int(0.9 * inst.q))
            if dec.all():
                Xo = st.U @ st.B + st.S.T
                assert rel(x_from(U1, B1, S1i, S1v, np.float64), Xo) <= TOL, target
                whole += 1
    finally:
        s.close()
    assert whole >= 1


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
        _, B1, S1i, S1v = s.get()              # b_k, s_k of iteration 6 (computed with U_5)
    finally:
        s.close()
    ks = np.sort(np.random.default_rng(17).choice(q, 8, replace=False))
    kt = torch.as_tensor(ks, device=dev.A.device)
    A = dev.A[kt].cpu().numpy()
    Y = dev.Y[kt].cpu().numpy()
    dev.free()
    st = state_from(U, B[:, ks], Si[ks], Sv[ks], n, 5, eta, np.float64)
    mg, _ = O.iterate_alg1(O.GaussianOperator(A), Y, st, rho)
    check_columns(st, mg, B1[:, ks], S1i[ks], S1v[ks], min_dec=6)


def test_one_step_fourier_128x128():
    from paper_2311_03824_gb300 import LRS_OP_DFT2D_MASK, Solver
    cfg = {k: v for k, v in C3.items() if k != "T"}
    inst = FourierInstance(**cfg)
    op = O.FourierOperator(inst.masks, inst.nx, inst.ny)
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, kind=LRS_OP_DFT2D_MASK,
               nx=inst.nx, ny=inst.ny)
    s.set_measurements(np.ascontiguousarray(inst.Y, np.complex64),
                       np.ascontiguousarray(inst.masks, np.int32))
    s.init()
    t = 0
    try:
        for target in (0, 30):
            s.iterate(target - t)
            t = target
            U, B, Si, Sv = s.get()
            eta, _ = s.progress()
            st = state_from(U, B, Si, Sv, inst.n, t, eta, np.complex128)
            mg, _ = O.iterate_alg1(op, inst.Y, st, inst.rho)
            s.iterate(1)
            t += 1
            U1, B1, S1i, S1v = s.get()
            dec = check_columns(st, mg, B1, S1i, S1v, min_dec=int(0.5 * inst.q))
            if dec.all():
                Xo = st.U @ st.B + st.S.T
                assert rel(x_from(U1, B1, S1i, S1v, np.complex128), Xo) <= TOL, target
    finally:
        s.close()
