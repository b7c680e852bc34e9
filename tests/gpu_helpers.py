"""Shared helpers of the GPU parity tests: run the CUDA solver through the C
ABI and the FP64 oracle on the same seeded instance, iterate by iterate.

FP32 arithmetic reproduces a HardThreshold decision of the FP64 oracle only
when the decision's margin (|v|_(rho) - |v|_(rho+1)) / max|v| exceeds the
relative error of the FP32 values v, about 1e-6 here; MARGIN_FP32 = 1e-4 is
the resolution the tests assume.  Columns whose oracle margin (the smallest
over the IHT sweeps of an iteration) is below it are "undecidable" for FP32.
"""
import numpy as np

import oracle.altgdmin_lrs as O

MARGIN_FP32 = 1e-4
TOL = 1e-5


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def oracle_run(inst, T, rho=None, **kw):
    rho = inst.rho if rho is None else rho
    return O.run_alg1(O.GaussianOperator(inst.A), inst.Y, inst.r, rho, T,
                      keep=tuple(range(T + 1)), Xstar=inst.Xstar, **kw)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def x_of(U, B, S_idx, S_val, q):
    X = U.astype(np.float64) @ B.astype(np.float64)
    for k in range(q):
        X[S_idx[k], k] += S_val[k]
    return X


def new_solver(inst, **opts):
    from paper_2311_03824_gb300 import Solver
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, **opts)
    s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                       np.ascontiguousarray(inst.A, np.float32))
    return s


def trajectory(inst, T, log, **solver_opts):
    """Run lrs_init + T x lrs_iterate(1); per iterate: relative X difference to
    the oracle, support mismatches among decidable columns, orthonormality."""
    s = new_solver(inst, **solver_opts)
    try:
        s.init()
        out = []
        undecided = np.zeros(inst.q, bool)      # a sub-resolution decision so far
        for t in range(T + 1):
            if t:
                s.iterate(1)
            U, B, S_idx, S_val = s.get()
            X = x_of(U, B, S_idx, S_val, inst.q)
            undecided |= log.margin[t] <= MARGIN_FP32
            ok = ~undecided
            bad = int(np.sum(np.any(np.sort(S_idx[ok], axis=1) != log.S_idx[t][ok], axis=1)))
            out.append(dict(t=t, rel=rel(X, log.X[t]), sup_bad=bad, undecided=int(undecided.sum()),
                            ortho=float(np.abs(U.T.astype(np.float64) @ U - np.eye(inst.r)).max()),
                            ascending=bool(np.all(np.diff(S_idx, axis=1) > 0)) if inst.rho > 1 else True))
        eta, _ = s.progress()
        return out, eta
    finally:
        s.close()


def one_step(inst, log, ts, **solver_opts):
    """From the oracle's iterate t (U_t, B_t, S_t, eta) run one GPU iteration
    and compare with the oracle's iterate t+1.  Returns per-t records."""
    s = new_solver(inst, **solver_opts)
    out = []
    try:
        for t in ts:
            U = np.ascontiguousarray(log.U[t].T, np.float32)           # n x r column-major
            B = np.ascontiguousarray(log.B[t].T, np.float32)           # r x q column-major
            Si = np.ascontiguousarray(log.S_idx[t], np.int32)
            Sv = np.ascontiguousarray(log.S_val[t], np.float32)
            from paper_2311_03824_gb300 import lrs as L
            L.lrs_set_state(s.h, U, B, Si, Sv, t, float(log.eta if t else 0.0))
            s.iterate(1)
            U1, B1, S_idx, S_val = s.get()
            X = x_of(U1, B1, S_idx, S_val, inst.q)
            dec = log.margin[t + 1] > MARGIN_FP32
            bad = int(np.sum(np.any(np.sort(S_idx[dec], axis=1) != log.S_idx[t + 1][dec], axis=1)))
            out.append(dict(t=t, rel=rel(X, log.X[t + 1]), sup_bad=bad,
                            undecided=int((~dec).sum())))
        return out
    finally:
        s.close()
