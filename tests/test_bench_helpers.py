"""Host-side arithmetic of bench.py against closed forms: the algorithmic
bytes of a Gaussian column-iteration, the flops of a 2D-DFT column-iteration,
the FP32 FMA peak from unit counts, and the workloads it accepts.  No GPU."""
import math
import subprocess
import sys

import pytest

import bench


def test_b_alg_matches_the_c1_and_c2_figures():
    # A_k once in float32, y_k, h_k, s_k (index + value), b_k
    assert bench.b_alg_per_col_iter(1000, 150, 5, 10) == 4 * 150 * 1000 + 4 * 150 + 4 * 1000 + 80 + 20
    assert bench.b_alg_per_col_iter(1000, 150, 5, 10) == 604_700
    # FP8 hi: one byte per element plus one FP32 row scale per row
    fp8 = bench.b_alg_per_col_iter(4096, 512, 10, 40, 1.0, 1)
    assert fp8 == 512 * 4096 + 4 * 512 + 4 * 512 + 4 * 4096 + 8 * 40 + 40
    # the stored-form bytes scale the A_k term only
    d = bench.b_alg_per_col_iter(4096, 512, 10, 40, 4.0) - bench.b_alg_per_col_iter(4096, 512, 10, 40, 2.0)
    assert d == 2 * 512 * 4096


def test_fourier_flops_closed_form():
    n, m, rho = 128 * 128, 2048, 82
    f = bench.fourier_flops_per_col_iter(n, m, rho)
    # three radix-2 2D FFTs (5 n log2 n each) and seven sparse DFTs of m x rho
    # complex multiply-adds (8 flops each)
    assert f == 3 * 5 * n * 14 + 7 * 8 * m * rho
    assert bench.fourier_flops_per_col_iter(n, m, 0) == 3 * 5 * n * math.log2(n)
    assert bench.fourier_flops_per_col_iter(n, m, rho, tau=1) == 5 * n * 14 + 3 * 8 * m * rho


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(80.54784)
    assert bench.fp32_peak_tflops(1000.0, nsm=1) == pytest.approx(0.256)


def test_bench_accepts_every_workload():
    out = subprocess.run([sys.executable, "bench.py", "--help"], capture_output=True, text=True,
                         cwd=bench.ROOT, timeout=120)
    assert out.returncode == 0
    for w in ("c1", "c2", "c3", "c4"):
        assert w in out.stdout
