"""Counter-based random numbers for the seeded synthetic inputs.

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11) gives four 32-bit words per (counter, key).  Gaussian
samples come from the Box-Muller transform of two 53-bit uniforms.  The
logarithm, sine and cosine used by Box-Muller are written out here from their
series (atanh series for log, Taylor series for sin/cos after quadrant
reduction) using only IEEE-754 double add, multiply, divide and square root,
each correctly rounded, so that a device implementation written to the same
definition reproduces every bit.

This module holds input generation only; it contains none of the solver's
arithmetic.
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)

TWO_M53 = 2.0 ** -53
TWO_26 = 2.0 ** 26
LN2 = 0.6931471805599453          # ln 2 rounded to double
SQRT_HALF = 0.7071067811865476    # 1/sqrt(2) rounded to double
HALF_PI = 1.5707963267948966      # pi/2 rounded to double


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: 4 uint64 arrays (values < 2**32), key: 2 uint64 scalars/arrays.
    Returns 4 uint64 arrays holding the 32-bit output words.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) for k in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _blocks(seed, tag, stream, first_block, nblocks):
    b = np.arange(first_block, first_block + nblocks, dtype=np.uint64)
    ctr = (b & MASK32, b >> np.uint64(32),
           np.full_like(b, np.uint64(stream) & MASK32),
           np.full_like(b, np.uint64(tag) & MASK32))
    key = (np.uint64(seed) & MASK32, (np.uint64(seed) >> np.uint64(32)) & MASK32)
    return philox4x32_10(ctr, key)


def _u53_open0(a, b):
    """(0, 1]: ((a>>5)*2^26 + (b>>6) + 1) * 2^-53."""
    return ((a >> np.uint64(5)).astype(np.float64) * TWO_26
            + (b >> np.uint64(6)).astype(np.float64) + 1.0) * TWO_M53


def _u53(a, b):
    """[0, 1): ((a>>5)*2^26 + (b>>6)) * 2^-53."""
    return ((a >> np.uint64(5)).astype(np.float64) * TWO_26
            + (b >> np.uint64(6)).astype(np.float64)) * TWO_M53


# 1/(2j+1), j = 0..11, each the correctly rounded double of the quotient.
_ATANH_C = [1.0 / (2 * j + 1) for j in range(12)]
# Taylor coefficients (-1)^j/(2j+1)! and (-1)^j/(2j)!, each a rounded double.
_SIN_C = []
_COS_C = []
_f = 1.0
for _j in range(0, 26):
    if _j:
        _f *= _j
    if _j % 2 == 1 and _j <= 25:
        _SIN_C.append((-1.0) ** ((_j - 1) // 2) / _f)
    if _j % 2 == 0 and _j <= 24:
        _COS_C.append((-1.0) ** (_j // 2) / _f)
del _f, _j


def ln_pos(u):
    """Natural log of u > 0: u = f 2^e, f in [1/sqrt2, sqrt2), ln f = 2 atanh t."""
    f, e = np.frexp(np.asarray(u, dtype=np.float64))
    low = f < SQRT_HALF
    f = np.where(low, f * 2.0, f)
    e = np.where(low, e - 1, e).astype(np.float64)
    t = (f - 1.0) / (f + 1.0)
    t2 = t * t
    s = np.full_like(t, _ATANH_C[-1])
    for c in reversed(_ATANH_C[:-1]):
        s = s * t2 + c
    return e * LN2 + (2.0 * t) * s


def sincos_turns(v):
    """sin(2 pi v), cos(2 pi v) for v in [0, 1) by quadrant reduction + Taylor."""
    v4 = np.asarray(v, dtype=np.float64) * 4.0
    qd = np.floor(v4)
    th = (v4 - qd) * HALF_PI
    t2 = th * th
    s = np.full_like(th, _SIN_C[-1])
    for c in reversed(_SIN_C[:-1]):
        s = s * t2 + c
    s = s * th
    c_ = np.full_like(th, _COS_C[-1])
    for c in reversed(_COS_C[:-1]):
        c_ = c_ * t2 + c
    qi = qd.astype(np.int64) & 3
    sin_o = np.select([qi == 0, qi == 1, qi == 2], [s, c_, -s], -c_)
    cos_o = np.select([qi == 0, qi == 1, qi == 2], [c_, -s, -c_], s)
    return sin_o, cos_o


def normals(seed, tag, stream, count, offset=0):
    """`count` N(0,1) doubles, elements offset..offset+count-1 of a stream.

    Element e uses Philox block e//2 of (seed, tag, stream); the block's words
    (x0,x1) give u1 in (0,1], (x2,x3) give u2 in [0,1); element 2b is
    sqrt(-2 ln u1) cos(2 pi u2) and element 2b+1 the matching sine.
    """
    if count == 0:
        return np.zeros(0)
    first = offset // 2
    last = (offset + count - 1) // 2
    x0, x1, x2, x3 = _blocks(seed, tag, stream, first, last - first + 1)
    u1 = _u53_open0(x0, x1)
    u2 = _u53(x2, x3)
    rad = np.sqrt(-2.0 * ln_pos(u1))
    sn, cs = sincos_turns(u2)
    z = np.empty(2 * len(u1))
    z[0::2] = rad * cs
    z[1::2] = rad * sn
    s0 = offset - 2 * first
    return z[s0:s0 + count]


def uniforms(seed, tag, stream, count):
    """`count` doubles in [0,1): two per Philox block ((x0,x1) then (x2,x3))."""
    if count == 0:
        return np.zeros(0)
    nb = (count + 1) // 2
    x0, x1, x2, x3 = _blocks(seed, tag, stream, 0, nb)
    u = np.empty(2 * nb)
    u[0::2] = _u53(x0, x1)
    u[1::2] = _u53(x2, x3)
    return u[:count]
