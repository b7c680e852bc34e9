"""What float32 arithmetic can resolve: the oracle's steps run in float32
against the same steps in float64.

HardThreshold (Algorithm 2, Section II-D) keeps the rho largest |v_i| of
v = s - mu g.  Its decision is decided by the gap
margin = (|v|_(rho) - |v|_(rho+1)) / max|v| (the oracle's `hard_threshold`).
A float32 evaluation of the same step computes v with a relative error of a
few float32 ulps and can legitimately keep another index when the gap is of
that size.  This study measures where that happens: from every logged FP64
iterate t of Algorithm 1 it runs one iteration (Algorithm 1, "Compute z_k,
M_k" to "U <- QR") in float32 and one in float64 from the same state, and
records, for every column, the FP64 step's smallest HardThreshold margin over
its IHT sweeps and whether the float32 step kept a different support.  The
initialisation (IHT from s = 0 with tau0 sweeps) is compared the same way.

It also measures how far float32 rounding moves the decision gap itself:
through the oracle's `perturb` hook (which here only records v and returns
it unchanged) it takes v of every IHT sweep of both steps and forms, per
column, the largest change of the gap between the float32 and float64 sweeps.
The GPU parity tests (tests/gpu_helpers.py) count a decision as decidable when
its FP64 margin exceeds both a floor MARGIN_FP32 = 1e-6 and ten times this
change, and the float32 step keeps the same support; the study reports what
that rule excludes on each instance.

The initialisation is different: its tau0 sweeps start from s = 0 and can
amplify a rounding difference until a decision with a large margin goes the
other way (the float32 departures with margins of 1e-2 below are all in the
initialisation).  Its supports are compared only on columns that the float32
probe finds decidable and that do not move when the FP64 initialisation is
rerun with rounding-size perturbations.

Run:  python tests/fp32_margin_study.py   (writes tests/golden/fp32_margin_study.txt)
It calls only the oracle and the input generators.  Test infrastructure.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle.altgdmin_lrs as O  # noqa: E402
from lrsgen import GaussianInstance  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "fp32_margin_study.txt")

# The instances of the GPU parity tests (small Gaussian workload, ragged slabs,
# tall columns, rank edges) and a column subset of the n=1000, m=150 workload.
INSTANCES = [
    ("n200_q200_r3_m80_rho4", dict(n=200, q=200, r=3, m=80, rho=4, seed=1), 300),
    ("n250_q40_r3_m36_rho3", dict(n=250, q=40, r=3, m=36, rho=3, seed=101), 20),
    ("n140_q24_r4_m300_rho5", dict(n=140, q=24, r=4, m=300, rho=5, seed=102), 8),
    ("n70_q30_r8_m40_rho6", dict(n=70, q=30, r=8, m=40, rho=6, seed=208), 12),
    ("n70_q30_r16_m48_rho2", dict(n=70, q=30, r=16, m=48, rho=2, seed=216), 12),
    ("n1000_q100_r5_m150_rho10", dict(n=1000, q=100, r=5, m=150, rho=10, seed=2), 40),
]


def cast_state(st, dt):
    return O.OracleState(U=st.U.astype(dt), B=st.B.astype(dt), S=st.S.astype(dt),
                         S_idx=st.S_idx.copy(), eta=st.eta, t=st.t)


def state_of(log, t, n):
    S = O.densify(log.S_idx[t], log.S_val[t], n)
    return O.OracleState(U=log.U[t].copy(), B=log.B[t].copy(), S=S, S_idx=log.S_idx[t].copy(),
                         eta=log.eta if t else None, t=t)


class Recorder:
    """perturb hook that records v of every IHT sweep and leaves it unchanged."""

    def __init__(self):
        self.v = []

    def __call__(self, v):
        self.v.append(np.array(v, dtype=np.float64))
        return v


def gap_change(r32, r64, rho):
    """Per column: largest change over the sweeps of the HardThreshold gap
    between the float32 and the float64 sweep."""
    d = np.zeros(r64.v[0].shape[0])
    for a, b in zip(r32.v, r64.v):
        ma = O.hard_threshold(a, rho)[2]
        mb = O.hard_threshold(b, rho)[2]
        ok = np.isfinite(ma) & np.isfinite(mb)
        d = np.maximum(d, np.where(ok, np.abs(ma - mb), 0.0))
    return d


def study(cfg, T):
    """Per column-step of every iteration t = 0..T-1: the FP64 step's smallest
    HardThreshold margin, whether the float32 step from the same state kept
    another support, and the float32 change of the gap; and for the
    initialisation the margins and departures alone."""
    inst = GaussianInstance(**cfg)
    op64 = O.GaussianOperator(inst.A)
    op32 = O.GaussianOperator(inst.A, np.float32)
    Y32 = inst.Y.astype(np.float32)
    _, log = O.run_alg1(op64, inst.Y, inst.r, inst.rho, T, keep=tuple(range(T + 1)))
    st64, _, _, m0 = O.init_alg1(op64, inst.Y, inst.r, inst.rho)
    st32, _, _, _ = O.init_alg1(op32, Y32, inst.r, inst.rho)
    init = (m0, np.any(st32.S_idx != st64.S_idx, axis=1))
    margins, departed, delta = [], [], []
    for t in range(T):
        r64, r32 = Recorder(), Recorder()
        st = state_of(log, t, inst.n)
        O.iterate_alg1(op64, inst.Y, st, inst.rho, perturb=r64)
        st = cast_state(state_of(log, t, inst.n), np.float32)
        O.iterate_alg1(op32, Y32, st, inst.rho, perturb=r32)
        margins.append(log.margin[t + 1])
        dep = np.any(st.S_idx != log.S_idx[t + 1], axis=1)
        departed.append(dep)
        delta.append(np.where(dep, np.nan, gap_change(r32, r64, inst.rho)))
    return (np.concatenate(margins), np.concatenate(departed), np.concatenate(delta)), init


MARGIN_FP32, DEC_FACTOR = 1e-6, 10.0     # the rule of the GPU parity tests


def summarise(name, steps, init):
    margins, departed, change = steps
    finite = np.isfinite(margins)
    dep = departed & finite
    worst = float(margins[dep].max()) if dep.any() else 0.0
    hist = []
    for lo in range(-9, 0):
        sel = finite & (margins >= 10.0 ** lo) & (margins < 10.0 ** (lo + 1))
        hist.append(f"1e{lo}:{int(sel.sum())}/{int((sel & departed).sum())}")
    c = change[np.isfinite(change)]
    excluded = ~((margins > MARGIN_FP32) & (margins > DEC_FACTOR * np.nan_to_num(change, nan=np.inf))
                 & ~departed)
    m0, d0 = init
    w0 = float(m0[d0 & np.isfinite(m0)].max()) if (d0 & np.isfinite(m0)).any() else 0.0
    return (f"{name} iteration_column_steps={margins.size} departed={int(departed.sum())} "
            f"max_departing_margin={worst:.3e} min_margin={np.min(margins):.3e} "
            f"gap_change_median={np.median(c):.2e} q99={np.quantile(c, 0.99):.2e} "
            f"max={c.max():.2e} excluded_by_rule={int(excluded.sum())} "
            f"decades(total/departed)={' '.join(hist)} | init_columns={m0.size} "
            f"init_departed={int(d0.sum())} init_max_departing_margin={w0:.3e}")


def main():
    lines = ["# float32 steps of Algorithm 1 against float64 steps from the same FP64 iterates",
             "# (tests/fp32_margin_study.py; oracle only).  max_departing_margin: the largest",
             "# FP64 HardThreshold margin at which the float32 step kept another support;",
             "# gap_change: how far float32 moved the decision gap (per column, largest over",
             "# the sweeps); excluded_by_rule: column-steps the parity tests' rule leaves out",
             f"# (margin <= {MARGIN_FP32:g}, margin <= {DEC_FACTOR:g} x gap_change, or departed)."]
    worst = 0.0
    for name, cfg, T in INSTANCES:
        steps, init = study(cfg, T)
        lines.append(summarise(name, steps, init))
        mg, dep, _ = steps
        d = dep & np.isfinite(mg)
        if d.any():
            worst = max(worst, float(mg[d].max()))
        print(lines[-1], flush=True)
    lines.append(f"iterations: max_departing_margin {worst:.3e}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(lines[-1])


if __name__ == "__main__":
    main()
