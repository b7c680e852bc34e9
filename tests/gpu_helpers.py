"""Shared helpers of the GPU parity tests: run the CUDA solver through the C
ABI and the FP64 oracle on the same seeded instance, iterate by iterate."""
import numpy as np

import oracle.altgdmin_lrs as O


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


def compare_trajectory(inst, T, log, margin_thr=1e-4, **solver_opts):
    """Per-iterate relative X difference and support agreement (columns whose
    oracle margin exceeds margin_thr) of the GPU run against the oracle log."""
    from paper_2311_03824_gb300 import Solver
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, **solver_opts)
    try:
        s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                           np.ascontiguousarray(inst.A, np.float32))
        s.init()
        out = []
        for t in range(T + 1):
            if t:
                s.iterate(1)
            U, B, S_idx, S_val = s.get()
            X = U.astype(np.float64) @ B.astype(np.float64)
            for k in range(inst.q):
                X[S_idx[k], k] += S_val[k]
            sel = log.margin[t] > margin_thr
            bad = int(np.sum(np.any(np.sort(S_idx[sel], axis=1) != log.S_idx[t][sel], axis=1)))
            out.append(dict(t=t, rel=rel(X, log.X[t]), sup_bad=bad, sup_checked=int(sel.sum()),
                            ortho=float(np.abs(U.T.astype(np.float64) @ U - np.eye(inst.r)).max()),
                            ascending=bool(np.all(np.diff(S_idx, axis=1) > 0)) if inst.rho > 1 else True))
        eta, tt = s.progress()
        return out, eta
    finally:
        s.close()
