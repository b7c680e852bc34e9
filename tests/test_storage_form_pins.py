"""Pins of the oracle's storage forms of A_k and of the defect-corrected
iteration (oracle/storage_forms.py) to things other than themselves:
library conversions (torch's bfloat16 and float8_e4m3fn casts, both round to
nearest even), the e4m3 format's closed form, rounding error bounds, and the
fixed-point property of the correction on exact data."""
import numpy as np
import pytest

import oracle.altgdmin_lrs as O
import oracle.storage_forms as F
from lrsgen import GaussianInstance

torch = pytest.importorskip("torch")


def test_bf16_round_matches_library_cast():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * np.exp2(rng.integers(-40, 40, 100000))).astype(np.float32)
    ties = ((x.view(np.uint32) & 0xFFFF0000) | 0x8000).view(np.float32)   # exact half-way cases
    x = np.concatenate([x, ties, np.float32([0.0, -0.0, 1.0, -3.5])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(F.bf16_round(x), ref)


def test_e4m3_value_set_closed_form():
    v = F.e4m3_values()
    assert len(v) == 127 and np.all(np.diff(v) > 0)
    assert v[0] == 0.0 and v[1] == 2.0 ** -9 and v[-1] == 448.0 == F.E4M3_MAX
    assert v[8] == 2.0 ** -6                                # smallest normal
    # every value is exactly representable in the library's e4m3 type
    back = torch.tensor(v, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float32)
    assert np.array_equal(back.numpy(), v.astype(np.float32))


def test_e4m3_round_matches_library_cast_and_saturates():
    v = F.e4m3_values()
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(100000) * np.exp2(rng.integers(-14, 9, 100000))).astype(np.float32)
    x = np.clip(x, -448, 448)
    mids = ((v[1:] + v[:-1]) / 2).astype(np.float32)        # ties: to the even code
    x = np.concatenate([x, mids, -mids])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(F.e4m3_round(x), ref)
    assert np.array_equal(F.e4m3_round(np.float32([500.0, -1e9, 449.0])), np.float32([448, -448, 448]))


def test_encode_error_bounds():
    A = GaussianInstance(n=300, q=6, r=2, m=40, rho=2, seed=3).A
    A64 = A.astype(np.float64)
    Ab, _ = F.encode(A, "bf16")
    assert np.all(np.abs(Ab - A64) <= 2.0 ** -8 * np.abs(A64))   # 8 significand bits
    Ah, s = F.encode(A, "fp8_hi")
    s1 = s[..., :1].astype(np.float64)
    # 3 mantissa bits: relative error <= 2^-4 of the normal range, plus half
    # the subnormal spacing (2^-10 in units of s1)
    assert np.all(np.abs(Ah - A64) <= 2.0 ** -4 * np.abs(A64) + 2.0 ** -10 * s1 * 1.0001)
    assert np.allclose(np.abs(A64).max(axis=2, keepdims=True), 448 * s1, rtol=1e-6)
    Ahl, s2 = F.encode(A, "fp8_hilo")
    assert np.array_equal(s2[..., :1], s[..., :1])
    e_hi, e_hl = np.abs(Ah - A64), np.abs(Ahl - A64)
    # the lo plane reduces the error by at least 2^4 relative to hi's largest error
    assert e_hl.max() <= e_hi.max() * 2.0 ** -4
    assert np.linalg.norm(Ahl - A64) < 0.05 * np.linalg.norm(Ah - A64)


def test_correction_fixed_point_on_exact_data():
    """With y_k = A_k x*_k exactly, ỹ(x*) = Ã_k x*_k: x* solves the corrected
    low-precision problem."""
    inst = GaussianInstance(n=120, q=10, r=2, m=50, rho=3, seed=4, y_float64=True)
    for form in ("bf16", "fp8_hi", "fp8_hilo"):
        At, _ = F.encode(inst.A, form)
        Yc = F.corrected_measurements(inst.A, At, inst.Y, inst.Xstar)
        AtX = (At.astype(np.float64) @ inst.Xstar.T[:, :, None])[:, :, 0]
        assert np.linalg.norm(Yc - AtX) <= 1e-13 * np.linalg.norm(inst.Y)


def test_defect_correction_recovers_exact_solution():
    """On a noiseless FP64 instance the corrected iteration on an FP8 operator
    reaches the exact solution, the uncorrected one stalls at the codec's
    error level."""
    inst = GaussianInstance(n=60, q=40, r=2, m=40, rho=2, seed=5, y_float64=True)
    At, _ = F.encode(inst.A, "fp8_hi")
    _, log = F.run_defect_corrected(inst.A, At, inst.Y, 2, 2, 120, 4, Xstar=inst.Xstar)
    assert log.err[-1] < 1e-10
    _, stale = F.run_defect_corrected(inst.A, At, inst.Y, 2, 2, 120, 10 ** 9, Xstar=inst.Xstar)
    assert stale.err[-1] > 1e-4
    # refine_every = 1 with Ã = A is plain Algorithm 1
    _, plain = O.run_alg1(O.GaussianOperator(inst.A), inst.Y, 2, 2, 30, Xstar=inst.Xstar)
    _, same = F.run_defect_corrected(inst.A, inst.A, inst.Y, 2, 2, 30, 1, Xstar=inst.Xstar)
    assert np.allclose(plain.err, same.err, rtol=1e-9, atol=1e-15)
