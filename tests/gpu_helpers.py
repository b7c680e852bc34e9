"""Shared helpers of the GPU parity tests: run the CUDA solver through the C
ABI and the FP64 oracle on the same seeded instance, iterate by iterate.

FP32 arithmetic reproduces a HardThreshold decision of the FP64 oracle only
when the decision's margin (|v|_(rho) - |v|_(rho+1)) / max|v| exceeds the
relative error of the FP32 values v, about 1e-6 here; MARGIN_FP32 = 1e-4 is
the resolution the tests assume.  Columns whose oracle margin (the smallest
over the IHT sweeps of an iteration) is below it are "undecidable" for FP32.

Margins do not capture every sensitivity: an IHT trajectory can itself
amplify rounding (for instance a mu that alternates between two values
from sweep to sweep), so that FP32 and FP64 leave a decision with a large
margin by different routes.  `step_sensitivity` / `run_sensitivity` measure
it directly: the oracle is rerun NPERT times with a relative perturbation
of 1e-7 (about a float32 ulp) applied to v = s - mu g before every
HardThreshold (the oracle's test hook), every column whose support moves
in any rerun is taken as undecidable, and the parity bar of an iterate
becomes max(1e-5, 10 x the largest relative change of X).
"""
import numpy as np

import oracle.altgdmin_lrs as O

MARGIN_FP32 = 1e-4
TOL = 1e-5
PERTURB = 1e-7
NPERT = 3


def rounding_noise(seed):
    """The oracle's perturb hook: v (1 + PERTURB N(0, 1)), seeded."""
    rng = np.random.default_rng(seed)
    return lambda v: v * (1.0 + PERTURB * rng.standard_normal(v.shape))


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


def trajectory(inst, T, log, sens=None, **solver_opts):
    """Run lrs_init + T x lrs_iterate(1); per iterate: relative X difference to
    the oracle, support mismatches among decidable columns, orthonormality.
    With `sens` (run_sensitivity) columns whose support moved under the
    perturbation are undecided and each record carries its bar."""
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
            bar = TOL
            if sens is not None:
                undecided |= sens[t][1]
                bar = max(TOL, 10.0 * sens[t][0])
            ok = ~undecided
            bad = int(np.sum(np.any(np.sort(S_idx[ok], axis=1) != log.S_idx[t][ok], axis=1)))
            out.append(dict(t=t, rel=rel(X, log.X[t]), sup_bad=bad, undecided=int(undecided.sum()),
                            bar=bar,
                            ortho=float(np.abs(U.T.astype(np.float64) @ U - np.eye(inst.r)).max()),
                            ascending=bool(np.all(np.diff(S_idx, axis=1) > 0)) if inst.rho > 1 else True))
        eta, _ = s.progress()
        return out, eta
    finally:
        s.close()


def state_of(log, t, n):
    """OracleState of the logged iterate t."""
    S = O.densify(log.S_idx[t], log.S_val[t], n)
    return O.OracleState(U=log.U[t].copy(), B=log.B[t].copy(), S=S, S_idx=log.S_idx[t].copy(),
                         eta=log.eta if t else None, t=t)


def step_sensitivity(op, y_of_t, log, ts, rho, n):
    """Per t: (largest relative change of X_{t+1}, columns whose support
    moves) over NPERT reruns of the oracle's step from iterate t with
    rounding-size perturbations inside the IHT."""
    out = {}
    for t in ts:
        d, moved = 0.0, np.zeros(log.S_idx[t].shape[0], bool)
        for i in range(NPERT):
            st = state_of(log, t, n)
            O.iterate_alg1(op, y_of_t(t), st, rho, perturb=rounding_noise(1000 * t + i))
            d = max(d, rel(st.U @ st.B + st.S.T, log.X[t + 1]))
            moved |= np.any(np.sort(st.S_idx, axis=1) != log.S_idx[t + 1], axis=1)
        out[t] = (d, moved)
    return out


def run_sensitivity(log, logs_p):
    """Per iterate of a run and its perturbed reruns: (largest relative change
    of X, columns whose support has moved at or before that iterate)."""
    out, moved = [], np.zeros(log.S_idx[0].shape[0], bool)
    for t in range(len(log.X)):
        d = 0.0
        for lp in logs_p:
            moved |= np.any(np.sort(lp.S_idx[t], axis=1) != log.S_idx[t], axis=1)
            d = max(d, rel(lp.X[t], log.X[t]))
        out.append((d, moved.copy()))
    return out


def one_step(inst, log, ts, sens=None, **solver_opts):
    """From the oracle's iterate t (U_t, B_t, S_t, eta) run one GPU iteration
    and compare with the oracle's iterate t+1.  Returns per-t records.  With
    `sens` (step_sensitivity) columns whose support moves under the
    perturbation count as undecided and the record carries the iterate's
    bar max(TOL, 10 x change)."""
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
            bar = TOL
            if sens is not None:
                dec = dec & ~sens[t][1]
                bar = max(TOL, 10.0 * sens[t][0])
            bad = int(np.sum(np.any(np.sort(S_idx[dec], axis=1) != log.S_idx[t + 1][dec], axis=1)))
            out.append(dict(t=t, rel=rel(X, log.X[t + 1]), sup_bad=bad,
                            undecided=int((~dec).sum()), bar=bar))
        return out
    finally:
        s.close()
