"""Fourier (row-masked 2D DFT) operator: CUDA solver against the FP64 oracle.

Same bars as the Gaussian parity tests (see gpu_helpers): one-step parity from
the oracle's iterates and trajectory parity up to the first HardThreshold
decision float32 cannot resolve."""
import numpy as np
import pytest

import oracle.altgdmin_lrs as O
from lrsgen import FourierInstance
from tests.gpu_helpers import MARGIN_FP32, TOL, gpu_available, rel

pytestmark = pytest.mark.gpu


def _solver(inst, **kw):
    from paper_2311_03824_gb300 import Solver, LRS_OP_DFT2D_MASK
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, kind=LRS_OP_DFT2D_MASK,
               nx=inst.nx, ny=inst.ny, **kw)
    s.set_measurements(np.ascontiguousarray(inst.Y, np.complex64),
                       np.ascontiguousarray(inst.masks, np.int32))
    return s


def _x(U, B, S_idx, S_val, q):
    X = U.astype(np.complex128) @ B.astype(np.complex128)
    for k in range(q):
        X[S_idx[k], k] += S_val[k]
    return X


def _oracle(inst, T):
    return O.run_alg1(O.FourierOperator(inst.masks, inst.nx, inst.ny), inst.Y, inst.r, inst.rho, T,
                      keep=tuple(range(T + 1)), Xstar=inst.Xstar)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


@pytest.mark.parametrize("nx,ny,m,rho", [(16, 16, 96, 4), (32, 16, 160, 6), (8, 32, 100, 3)])
def test_fourier_one_step_parity(nx, ny, m, rho):
    inst = FourierInstance(nx=nx, ny=ny, q=12, r=2, m=m, rho=rho, seed=41, center=4)
    T = 10
    _, log = _oracle(inst, T)
    s = _solver(inst)
    from paper_2311_03824_gb300 import lrs as L
    checked = 0
    for t in range(T):
        U = np.ascontiguousarray(log.U[t].T, np.complex64)
        B = np.ascontiguousarray(log.B[t].T, np.complex64)
        Si = np.ascontiguousarray(log.S_idx[t], np.int32)
        Sv = np.ascontiguousarray(log.S_val[t], np.complex64)
        L.lrs_set_state(s.h, U, B, Si, Sv, t, float(log.eta if t else 0.0))
        s.iterate(1)
        U1, B1, S_idx, S_val = s.get()
        dec = log.margin[t + 1] > MARGIN_FP32
        assert np.all(np.sort(S_idx[dec], 1) == log.S_idx[t + 1][dec]), t
        if dec.all():
            assert rel(_x(U1, B1, S_idx, S_val, inst.q), log.X[t + 1]) <= TOL, t
            checked += 1
    s.close()
    assert checked >= T // 2


def test_fourier_trajectory_and_init():
    inst = FourierInstance(nx=16, ny=16, q=16, r=2, m=100, rho=4, seed=42, center=4)
    T = 25
    _, log = _oracle(inst, T)
    s = _solver(inst)
    s.init()
    undecided = np.zeros(inst.q, bool)
    for t in range(T + 1):
        if t:
            s.iterate(1)
        U, B, S_idx, S_val = s.get()
        X = _x(U, B, S_idx, S_val, inst.q)
        undecided |= log.margin[t] <= MARGIN_FP32
        ok = ~undecided
        assert np.all(np.sort(S_idx[ok], 1) == log.S_idx[t][ok]), t
        if not undecided.any():
            assert rel(X, log.X[t]) <= TOL, (t, rel(X, log.X[t]))
        assert np.abs(U.conj().T @ U - np.eye(inst.r)).max() < 1e-5
    eta, _ = s.progress()
    assert abs(eta - log.eta) <= 1e-4 * log.eta
    s.close()
