"""Shared helpers of the GPU parity tests: run the CUDA solver through the C
ABI and the FP64 oracle on the same seeded instance, step by step.

Which HardThreshold decisions are compared.  FP32 arithmetic reproduces a
decision of the FP64 oracle only when the decision's gap
margin = (|v|_(rho) - |v|_(rho+1)) / max|v| (Algorithm 2; the oracle's
`hard_threshold`) exceeds what float32 rounding moves it by.  Every compared
step is therefore probed: besides the FP64 oracle step, the same oracle step
is run in float32 from the same state (the oracle's operators take a dtype),
and a column's decision counts as decidable when
  * its FP64 margin (smallest over the IHT sweeps) exceeds MARGIN_FP32 = 1e-6,
  * it exceeds DEC_FACTOR = 10 times the change of the margin between the
    float32 and float64 steps (largest over the sweeps), and
  * the float32 step keeps the same support.
tests/fp32_margin_study.py (results in tests/golden/fp32_margin_study.txt)
measures this on the instances of these tests: no float32 step departed from
the FP64 support at any margin (the smallest margin seen is 2.5e-6), the
median change of the gap is 6e-8 to 3e-6 and its 99th percentile 3e-6 to
2e-3, and the rule leaves out 1 of 65,712 column-steps; so the floor sits at
the float32 resolution and the per-column factor covers the columns whose mu is badly conditioned.  The initialisation's tau0 sweeps from
s = 0 can amplify a rounding difference past large margins; its decisions
are in addition rerun NPERT times with a relative perturbation of PERTURB
(about a float32 ulp) applied to v before each HardThreshold (the oracle's
test hook), and columns that move are not compared.

What is compared.  b_k and s_k of a step depend only on column k and U_t, so
they are compared on every decidable column (supports identical, values
within TOL relative over those columns); X_{t+1} = U_{t+1} B_{t+1} + S_{t+1}
mixes all columns through the gradient and is compared as a whole (TOL)
whenever every column is decidable.  Each test bounds the share of column-
steps it excludes (MAX_EXCLUDED) and the number of whole-X checks it must
make.
"""
import json
import os

import numpy as np

import oracle.altgdmin_lrs as O

MARGIN_FP32 = 1e-6
DEC_FACTOR = 10.0
TOL = 1e-5
DEV_FACTOR = 10.0
BAR_CAP = 1e-3
MAX_EXCLUDED = 0.01
PERTURB = 1e-7
NPERT = 3


def rounding_noise(seed):
    """The oracle's perturb hook: v (1 + PERTURB N(0, 1)), seeded."""
    rng = np.random.default_rng(seed)
    return lambda v: v * (1.0 + PERTURB * rng.standard_normal(v.shape))


class Recorder:
    """perturb hook that records v of every IHT sweep and returns it unchanged."""

    def __init__(self):
        self.v = []

    def __call__(self, v):
        self.v.append(np.array(v, copy=True))
        return v


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------- problems --

class Problem:
    """Oracle side of one instance: the FP64 operator, its float32 twin and the
    measurements the solver sees."""

    def __init__(self, op64, op32, Y, r, rho, A=None):
        self.op64, self.op32 = op64, op32
        self.A = A          # the Gaussian operator's stored values (row orders of the probe)
        self.Y = np.asarray(Y)
        self.n, self.q, self.r, self.rho = op64.n, op64.q, r, rho
        self.cplx = op64.complex
        self.dt = np.complex128 if self.cplx else np.float64

    @staticmethod
    def gaussian(inst, A=None, rho=None):
        A = inst.A if A is None else A
        return Problem(O.GaussianOperator(A), O.GaussianOperator(A, np.float32), inst.Y,
                       inst.r, inst.rho if rho is None else rho, A=np.asarray(A))

    @staticmethod
    def fourier(inst, rho=None):
        return Problem(O.FourierOperator(inst.masks, inst.nx, inst.ny),
                       O.FourierOperator(inst.masks, inst.nx, inst.ny, np.complex64),
                       inst.Y, inst.r, inst.rho if rho is None else rho)

    def y32(self, Y):
        return np.asarray(Y).astype(np.complex64 if self.cplx else np.float32)


def oracle_run(inst, T, rho=None, **kw):
    rho = inst.rho if rho is None else rho
    return O.run_alg1(O.GaussianOperator(inst.A), inst.Y, inst.r, rho, T,
                      keep=tuple(range(T + 1)), Xstar=inst.Xstar, **kw)


def x_of(U, B, S_idx, S_val, q):
    dt = np.complex128 if np.iscomplexobj(U) else np.float64
    X = U.astype(dt) @ B.astype(dt)
    for k in range(q):
        X[S_idx[k], k] += S_val[k]
    return X


def sorted_support(S_idx, S_val):
    o = np.argsort(S_idx, axis=1)
    return np.take_along_axis(S_idx, o, 1).astype(np.int64), np.take_along_axis(S_val, o, 1)


def state_of(log, t, n):
    """OracleState of the logged oracle iterate t."""
    S = O.densify(log.S_idx[t], log.S_val[t], n)
    return O.OracleState(U=log.U[t].copy(), B=log.B[t].copy(), S=S, S_idx=log.S_idx[t].copy(),
                         eta=log.eta if t else None, t=t)


def state_from_gpu(g, n, t, eta, dt):
    """OracleState (FP64 or complex128) of a GPU iterate g = (U n x r, B r x q,
    S_idx q x rho, S_val q x rho)."""
    U, B, S_idx, S_val = g
    q = B.shape[1]
    Si, Sv = sorted_support(S_idx, S_val)
    S = np.zeros((q, n), dt)
    if Si.size:
        np.put_along_axis(S, Si, Sv.astype(dt), axis=1)
    return O.OracleState(U=U.astype(dt), B=B.astype(dt), S=S, S_idx=Si,
                         eta=eta if t else None, t=t)


def cast_state(st, dt):
    return O.OracleState(U=st.U.astype(dt), B=st.B.astype(dt), S=st.S.astype(dt),
                         S_idx=st.S_idx.copy(), eta=st.eta, t=st.t)


def _gap_change(r32, r64, rho):
    """Per column: largest change over the IHT sweeps of the HardThreshold gap
    between the float32 and float64 sweeps (recorded v per sweep)."""
    d = np.zeros(r64.v[0].shape[0]) if r64.v else None
    for a, b in zip(r32.v, r64.v):
        ma = O.hard_threshold(a, rho)[2]
        mb = O.hard_threshold(b, rho)[2]
        ok = np.isfinite(ma) & np.isfinite(mb)     # (no gap when rho = n)
        diff = np.zeros_like(d)
        diff[ok] = np.abs(ma[ok] - mb[ok])
        d = np.maximum(d, diff)
    return d


def _sub_state(st, ks, dt):
    return O.OracleState(U=st.U.astype(dt), B=st.B[:, ks].astype(dt), S=st.S[ks].astype(dt),
                         S_idx=st.S_idx[ks].copy(), eta=st.eta, t=st.t)


def _probe_columns(P, st, Y, ks, mg, r64=None):
    """Decidable among columns ks: the FP64 and float32 steps of those columns
    from state st (their supports, b_k and s_k depend only on the column and
    U_t), sweep by sweep.  r64: the recorded FP64 sweeps when the caller's
    step already covered exactly these columns."""
    a = None
    if r64 is None:
        r64 = Recorder()
        a = _sub_state(st, ks, P.dt)
        O.iterate_alg1(P.op64.subset(ks), Y[ks], a, P.rho, perturb=r64)
    r32 = Recorder()
    b = _sub_state(st, ks, np.complex64 if P.cplx else np.float32)
    O.iterate_alg1(P.op32.subset(ks), P.y32(Y[ks]), b, P.rho, perturb=r32)
    return b, r32, r64, a


NORDERS = 3


def _row_order_deviations(P, st, Y, st64, dec):
    """The float32 step again with the rows of every A_k and y_k taken in
    other orders (a symmetry of the problem: the step is the same in exact
    arithmetic, its float32 sums over the rows are not), NORDERS times: the
    deviations from the FP64 step, so that a step's bar reflects the spread
    of float32 evaluations rather than the one order numpy uses."""
    if P.A is None:
        return []
    out = []
    m = P.A.shape[1]
    for i in range(NORDERS):
        pi = np.random.default_rng(4099 + i).permutation(m)
        op = O.GaussianOperator(P.A[:, pi, :], np.float32)
        b = cast_state(st, np.float32)
        O.iterate_alg1(op, P.y32(np.asarray(Y)[:, pi]), b, P.rho)
        if np.all(b.S_idx[dec] == st64.S_idx[dec]):
            out.append(_deviation(b, st64, dec))
    return out


def _deviation(st32, st64, dec):
    """How far the float32 step lies from the FP64 step on the decidable
    columns: relative differences of b_k, s_k, the whole X (when every column
    is decidable) and eta."""
    d = dict(b=0.0, s=0.0, x=0.0, eta=0.0)
    if dec.any():
        d["b"] = rel(st32.B[:, dec].astype(st64.B.dtype), st64.B[:, dec])
        if st64.S_idx.shape[1]:
            So = np.take_along_axis(st64.S[dec], st64.S_idx[dec], 1)
            S3 = np.take_along_axis(st32.S[dec], st32.S_idx[dec], 1).astype(So.dtype)
            d["s"] = rel(S3, So) if np.linalg.norm(So) > 0 else 0.0
    if dec.all():
        d["x"] = rel((st32.U.astype(st64.U.dtype) @ st32.B.astype(st64.B.dtype) + st32.S.T),
                     st64.U @ st64.B + st64.S.T)
    if st64.eta:
        d["eta"] = abs(float(st32.eta) - st64.eta) / st64.eta
    return d


def probe_step(P, st, Y=None, sens=0, chunk=None):
    """The FP64 oracle step from state `st` (not modified) and its float32
    probe.  Returns (FP64 state after the step, FP64 margins, decidable,
    float32 deviation).  chunk: columns per batch (memory of large problems;
    the deviation of the whole X and eta is then not measured)."""
    Y = np.asarray(P.Y if Y is None else Y)
    st64 = cast_state(st, P.dt)
    whole = chunk is None or chunk >= P.q
    rec = Recorder() if whole else None
    mg, _ = O.iterate_alg1(P.op64, Y, st64, P.rho, chunk=chunk, perturb=rec)
    step = P.q if whole else chunk
    dec = mg > MARGIN_FP32
    dev = dict(b=0.0, s=0.0, x=0.0, eta=0.0)
    for k0 in range(0, P.q, step):
        ks = np.arange(k0, min(P.q, k0 + step))
        st32, r32, r64, _ = _probe_columns(P, st, Y, ks, mg, rec)
        dec[ks] &= np.all(st32.S_idx == st64.S_idx[ks], axis=1)
        if r64.v:
            dec[ks] &= mg[ks] > DEC_FACTOR * _gap_change(r32, r64, P.rho)
        if whole:
            dev = _deviation(st32, st64, dec)
            for d2 in _row_order_deviations(P, st, Y, st64, dec):
                dev = {q: max(dev[q], d2[q]) for q in dev}
    for i in range(sens):
        sp = cast_state(st, P.dt)
        O.iterate_alg1(P.op64, Y, sp, P.rho, perturb=rounding_noise(7919 * st.t + i), chunk=chunk)
        dec &= np.all(sp.S_idx == st64.S_idx, axis=1)
    return st64, mg, dec, dev


def probe_init(P, sens=NPERT):
    """The FP64 initialisation, its float32 probe and NPERT perturbed reruns.
    Returns (FP64 initial state, margins, decidable)."""
    r64, r32 = Recorder(), Recorder()
    st64, _, _, mg = O.init_alg1(P.op64, P.Y, P.r, P.rho, perturb=r64)
    st32, _, _, _ = O.init_alg1(P.op32, P.y32(P.Y), P.r, P.rho, perturb=r32)
    dec = (mg > MARGIN_FP32) & np.all(st32.S_idx == st64.S_idx, axis=1)
    if r64.v:
        dec &= mg > DEC_FACTOR * _gap_change(r32, r64, P.rho)
    for i in range(sens):
        sp, _, _, _ = O.init_alg1(P.op64, P.Y, P.r, P.rho, perturb=rounding_noise(104729 + i))
        dec &= np.all(sp.S_idx == st64.S_idx, axis=1)
    return st64, mg, dec


def bars(dev, tol=TOL):
    """Per-quantity bars of one step: TOL, or DEV_FACTOR times what float32
    arithmetic itself departs from FP64 on this step (the float32 probe),
    whichever is larger, capped at BAR_CAP."""
    dev = dev or {}
    return {q: min(BAR_CAP, max(tol, DEV_FACTOR * dev.get(q, 0.0))) for q in ("b", "s", "x")}


def compare_step(st64, dec, g_next, tol=TOL, basis_free=False, whole=True, dev=None):
    """GPU iterate g_next = (U, B, S_idx, S_val) against the FP64 oracle state
    st64 of the same step on the decidable columns (and as a whole when all
    are).  basis_free: compare the low-rank columns U b_k instead of b_k (the
    initialisation, where U0 is the same subspace in another basis).
    whole=False: columns sampled from a larger problem (no whole-X check).
    dev: the float32 probe's deviation of this step (see `bars`)."""
    U1, B1, S1i, S1v = g_next
    q = B1.shape[1]
    Si, Sv = sorted_support(S1i, S1v)
    out = dict(excluded=int((~dec).sum()), columns=q, sup_bad=0, b_rel=0.0, s_rel=0.0,
               whole=None, ascending=True, bar=bars(dev, tol))
    out["raised"] = any(v > tol for v in out["bar"].values())
    if st64.S_idx.shape[1] > 1:
        out["ascending"] = bool(np.all(np.diff(S1i, axis=1) > 0))
    if dec.any():
        out["sup_bad"] = int(np.sum(np.any(Si[dec] != st64.S_idx[dec], axis=1)))
        if basis_free:
            out["b_rel"] = rel(U1.astype(st64.U.dtype) @ B1[:, dec].astype(st64.B.dtype),
                               st64.U @ st64.B[:, dec])
        else:
            out["b_rel"] = rel(B1[:, dec].astype(st64.B.dtype), st64.B[:, dec])
        if Si.shape[1]:
            So = np.take_along_axis(st64.S[dec], st64.S_idx[dec], 1)
            out["s_rel"] = rel(Sv[dec].astype(So.dtype), So) if np.linalg.norm(So) > 0 else 0.0
    if whole and dec.all():
        Xo = st64.U @ st64.B + st64.S.T
        out["whole"] = rel(x_of(U1, B1, S1i, S1v, q), Xo)
    out["ortho"] = float(np.abs(U1.conj().T.astype(np.complex128) @ U1 - np.eye(U1.shape[1])).max())
    out["tol"] = tol
    return out


def check_records(recs, min_whole, max_excluded=MAX_EXCLUDED):
    """Assert the per-step records of a parity test and return its summary:
    supports identical and b_k, s_k within the step's bars on decidable
    columns, whole X within its bar where every column is decidable (at
    least min_whole such steps), excluded column-steps at most max_excluded
    of all.  The summary counts the steps whose bar float32 itself raised
    above TOL."""
    whole = 0
    excl = sum(r["excluded"] for r in recs)
    tot = sum(r["columns"] for r in recs)
    for r in recs:
        b = r["bar"]
        assert r["sup_bad"] == 0, ("support mismatch on decidable columns", r)
        assert r["b_rel"] <= b["b"], ("b_k", r)
        assert r["s_rel"] <= b["s"], ("s_k", r)
        assert r["ascending"], r
        assert r["ortho"] < 1e-5, r
        if r["whole"] is not None:
            assert r["whole"] <= b["x"], ("X", r)
            whole += 1
    assert whole >= min_whole, ("whole-X checks", whole, min_whole)
    assert excl <= max_excluded * tot, ("excluded column-steps", excl, tot)
    summary = dict(steps=len(recs), whole=whole, excluded=excl, column_steps=tot,
                   raised=sum(1 for r in recs if r["raised"]),
                   max_b=max((r["b_rel"] for r in recs), default=0.0),
                   max_s=max((r["s_rel"] for r in recs), default=0.0),
                   max_x=max((r["whole"] for r in recs if r["whole"] is not None), default=0.0))
    log = os.environ.get("LRS_PARITY_LOG")
    if log:                      # one JSON line per checked run (the excluded shares)
        with open(log, "a") as f:
            f.write(json.dumps(dict(test=os.environ.get("PYTEST_CURRENT_TEST", ""), **summary)) + "\n")
    return summary


# ----------------------------------------------------------- GPU runs --

def new_solver(inst, **opts):
    from paper_2311_03824_gb300 import Solver
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, **opts)
    s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                       np.ascontiguousarray(inst.A, np.float32))
    return s


def new_fourier_solver(inst, **opts):
    from paper_2311_03824_gb300 import LRS_OP_DFT2D_MASK, Solver
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, kind=LRS_OP_DFT2D_MASK,
               nx=inst.nx, ny=inst.ny, **opts)
    s.set_measurements(np.ascontiguousarray(inst.Y, np.complex64),
                       np.ascontiguousarray(inst.masks, np.int32))
    return s


def set_gpu_state(s, st, cplx):
    """Load an oracle state into the solver (lrs_set_state)."""
    from paper_2311_03824_gb300 import lrs as L
    ct = np.complex64 if cplx else np.float32
    U = np.ascontiguousarray(st.U.T, ct)           # n x r column-major
    B = np.ascontiguousarray(st.B.T, ct)           # r x q column-major
    Si = np.ascontiguousarray(st.S_idx, np.int32)
    Sv = np.ascontiguousarray(np.take_along_axis(st.S, st.S_idx, 1) if st.S_idx.size
                              else np.zeros(st.S_idx.shape), ct)
    L.lrs_set_state(s.h, U, B, Si, Sv, st.t, float(st.eta or 0.0))


def one_step(P, s, log, ts, y_of_t=None, tol=TOL):
    """From the oracle's iterate t (lrs_set_state) one GPU iteration, compared
    with the probed FP64 oracle step from the same state."""
    recs = []
    for t in ts:
        st = state_of(log, t, P.n)
        Y = None if y_of_t is None else y_of_t(t)
        st64, _, dec, dev = probe_step(P, st, Y)
        set_gpu_state(s, st, P.cplx)
        s.iterate(1)
        r = compare_step(st64, dec, s.get(), tol, dev=dev)
        r["t"] = t
        recs.append(r)
    return recs


def gpu_trajectory(s, T):
    """lrs_init, then T x lrs_iterate(1): the GPU iterates t = 0..T and eta."""
    s.init()
    states = [s.get()]
    for _ in range(T):
        s.iterate(1)
        states.append(s.get())
    eta, _ = s.progress()
    return states, eta


def init_record(P, g0, tol=TOL):
    """The GPU initialisation g0 = (U0, B0, S_idx, S_val) against the oracle's
    (Algorithm 1, Initialization).  The IHT supports and values are compared
    on the columns the probe finds decidable.  U0 and b_k depend on every
    column through L0, so they are compared with what the oracle computes
    from the GPU's own supports: U0 against the top-r left singular subspace
    of L0 = [A_k^H (y_k - A_k s_k)] (FP64, full SVD; 1 - cos of the principal
    angles below 1e-6), and b_k against (A_k U0)^+ (y_k - A_k s_k) (FP64
    pseudo-inverse, relative TOL over all columns)."""
    st0, _, dec = probe_init(P)
    rec = compare_step(st0, dec, g0, tol, whole=False)
    rec["b_rel"] = 0.0
    U, B, S_idx, S_val = g0
    gs = state_from_gpu(g0, P.n, 0, None, P.dt)
    R = np.asarray(P.Y, P.dt) - P.op64.A(gs.S)
    L0 = P.op64.AH(R).T
    Ut, _ = O.top_r_left(L0, P.r)
    cos = np.linalg.svd(U.astype(P.dt).conj().T @ Ut, compute_uv=False)
    rec["u0_angle"] = float(np.max(np.abs(1.0 - cos)))
    assert rec["u0_angle"] < 1e-6, ("U0 subspace", rec["u0_angle"])
    Bo = O.pinv_apply(P.op64.AU(U.astype(P.dt)), R).T
    rec["b0_rel"] = rel(B.astype(P.dt), Bo)
    assert rec["b0_rel"] <= tol, ("b_k of the initialisation", rec["b0_rel"])
    rec["t"] = 0
    return rec


def trajectory_records(P, states, eta, init_check=True, tol=TOL):
    """Every step of a GPU trajectory against the probed FP64 oracle step from
    the GPU's own previous iterate; the first record compares the GPU
    initialisation with the oracle's (when init_check)."""
    recs = [init_record(P, states[0], tol)] if init_check else []
    for t in range(len(states) - 1):
        st = state_from_gpu(states[t], P.n, t, eta, P.dt)
        st64, _, dec, dev = probe_step(P, st)
        r = compare_step(st64, dec, states[t + 1], tol, dev=dev)
        if t == 0:   # eta of the first step against the oracle's from the same state
            r["eta_rel"] = abs(eta - st64.eta) / st64.eta
            assert r["eta_rel"] <= max(1e-6, DEV_FACTOR * dev["eta"]), ("eta", r["eta_rel"])
        r["t"] = t + 1
        recs.append(r)
    return recs


def trajectory_agreement(states, log):
    """Relative X difference between the GPU trajectory and the oracle's own
    trajectory at every t, and the first t at which a support differs."""
    q = states[0][1].shape[1]
    rels, first = [], None
    for t, g in enumerate(states):
        rels.append(rel(x_of(*g, q), log.X[t]))
        if first is None and np.any(sorted_support(g[2], g[3])[0] != log.S_idx[t]):
            first = t
    return rels, first
