"""Storage forms of the Gaussian operator A_k and the defect-corrected
iteration that runs on them.

TEST INFRASTRUCTURE, like the rest of `oracle/`: only the tests, the smoke
check and the benchmark's CPU-baseline leg may import it.

The paper computes in one precision throughout; these forms are the
solver's reduced-storage options, defined here from first principles:

  * BF16: every element rounded to the nearest bfloat16 (8 significand
    bits, ties to even).
  * FP8 hi (e4m3 with a row scale): s1_i = max_j |A(i, j)| / 448 (448 is the
    largest finite e4m3 value; an all-zero row takes s1_i = 1), and
    hi(i, j) = e4m3(A(i, j) / s1_i), decoded as s1_i * hi(i, j).
  * FP8 hi/lo: as above, plus lo(i, j) = e4m3(res(i, j) / s2_i) of the
    remainder res = A - s1_i hi with its own scale
    s2_i = max_j |res(i, j)| / 448, decoded as s1_i hi + s2_i lo.
  e4m3 rounding is to the nearest representable value, ties to the even
  code, saturating at +-448.  Scales, quotients and the remainder are
  single-precision operations (each result rounded to float32), the decoded
  sum s2 lo + s1 hi is rounded once.

Defect correction: with the exact operator A_k and its stored form Ã_k, the
corrected measurements at the iterate x_k = U b_k + s_k are
ỹ_k = y_k - (A_k - Ã_k) x_k; an iteration on (Ã_k, ỹ_k) then has every exact
solution of y_k = A_k x_k as a fixed point.  ỹ is refreshed before the first
iteration and then every `refine_every` iterations.
"""
from __future__ import annotations

import numpy as np

from . import altgdmin_lrs as O

E4M3_MAX = 448.0


def bf16_round(a):
    """float32 -> nearest bfloat16 value (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    v = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return v.view(np.float32)


def e4m3_values():
    """The 127 non-negative finite e4m3 values, indexed by their code 0..126
    (code = 8 * exponent field + mantissa field; exponent bias 7; exponent
    field 0 is subnormal, m/8 * 2^-6; code 127 is NaN)."""
    vals = []
    for code in range(127):
        e, mnt = code >> 3, code & 7
        vals.append(mnt / 8.0 * 2.0 ** -6 if e == 0 else (1.0 + mnt / 8.0) * 2.0 ** (e - 7))
    return np.array(vals, np.float64)


_E4M3 = e4m3_values()


def e4m3_round(x):
    """Nearest e4m3 value of float32 x (ties to the even code), saturated at
    +-448; returned as float32 (exact)."""
    x = np.asarray(x, np.float32).astype(np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    hi = np.clip(np.searchsorted(_E4M3, a, side="left"), 0, 126)  # first value >= a
    lo = np.maximum(hi - 1, 0)
    dlo, dhi = a - _E4M3[lo], _E4M3[hi] - a
    pick = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo % 2 == 0, lo, hi)))
    pick = np.where(_E4M3[hi] == a, hi, pick)
    return (np.sign(x) * _E4M3[pick]).astype(np.float32)


def _f32(v):
    return np.asarray(v, np.float32)


def encode(A, form):
    """Decoded stored form of A (q, m, n) float32 -> (Ã float32, scales).
    form: "bf16", "fp8_hi" or "fp8_hilo".  scales: (q, m, 1 or 2) float32."""
    A = _f32(A)
    if form == "bf16":
        return bf16_round(A), None
    amax = np.abs(A).max(axis=2, keepdims=True)
    s1 = np.where(amax > 0, _f32(amax / np.float32(E4M3_MAX)), np.float32(1.0)).astype(np.float32)
    hi = e4m3_round(_f32(A / s1))
    dec_hi = _f32(hi * s1)
    if form == "fp8_hi":
        return dec_hi, s1
    if form != "fp8_hilo":
        raise ValueError(form)
    # the residual A - s1 * hi taken exactly (float64 holds the product and the
    # difference without rounding) and rounded once to float32
    res = _f32(A.astype(np.float64) - hi.astype(np.float64) * s1.astype(np.float64))
    rmax = np.abs(res).max(axis=2, keepdims=True)
    s2 = np.where(rmax > 0, _f32(rmax / np.float32(E4M3_MAX)), np.float32(1.0)).astype(np.float32)
    lo = e4m3_round(_f32(res / s2))
    dec = _f32(lo.astype(np.float64) * s2.astype(np.float64) + dec_hi.astype(np.float64))
    return dec, np.concatenate([s1, s2], axis=2)


def corrected_measurements(A, At, Y, X):
    """ỹ_k = y_k - (A_k - Ã_k) x_k for every column (X: n x q), in float64."""
    D = np.asarray(A, np.float64) - np.asarray(At, np.float64)
    return np.asarray(Y, np.float64) - (D @ X.T[:, :, None])[:, :, 0]


def run_defect_corrected(A, At, Y, r, rho, T, refine_every, Xstar=None, keep=(), tau0=10,
                         tau=3, c_eta=0.14, perturb=None):
    """Algorithm 1 on the stored form Ã with defect correction: the
    initialisation runs on (Ã, y); iteration t + 1 runs on (Ã, ỹ) with ỹ
    recomputed from the iterate X_t when t is 0 or a multiple of
    refine_every.  Logs as `run_alg1` (err against Xstar every t).
    perturb: see altgdmin_lrs.iht (test aid, None in plain runs)."""
    opt = O.GaussianOperator(At)
    st, _, sv, m0 = O.init_alg1(opt, Y, r, rho, tau0, perturb=perturb)
    log = O.OracleLog()
    log.init_sv = sv

    def record(t, margin):
        X = st.U @ st.B + st.S.T
        if Xstar is not None:
            log.t.append(t)
            log.err.append(O.relative_error(X, Xstar))
        if t in keep:
            log.X.append(X.copy())
            log.U.append(st.U.copy())
            log.B.append(st.B.copy())
            log.S_idx.append(st.S_idx.copy())
            log.S_val.append(np.take_along_axis(st.S, st.S_idx, axis=1) if st.S_idx.size
                             else np.zeros((opt.q, 0)))
            log.margin.append(margin.copy())

    record(0, m0)
    Yc = None
    for t in range(T):
        if t % refine_every == 0:
            Yc = corrected_measurements(A, At, Y, st.U @ st.B + st.S.T)
        mg, _ = O.iterate_alg1(opt, Yc, st, rho, tau, c_eta, perturb=perturb)
        record(st.t, mg)
    log.eta = st.eta
    return st, log
