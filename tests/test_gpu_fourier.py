"""Fourier (row-masked 2D DFT) operator: CUDA solver against the FP64 oracle.

Same bars as the Gaussian parity tests (tests/gpu_helpers.py): one-step
parity from the oracle's iterates, and every step of a GPU trajectory
against the probed oracle step from the GPU's own previous iterate (eta of
the first step included)."""
import numpy as np
import pytest

import oracle.altgdmin_lrs as O
from lrsgen import FourierInstance
from tests.gpu_helpers import (TOL, Problem, check_records, gpu_available, gpu_trajectory,
                               new_fourier_solver, one_step, trajectory_agreement,
                               trajectory_records)

pytestmark = pytest.mark.gpu


def _oracle(inst, T):
    return O.run_alg1(O.FourierOperator(inst.masks, inst.nx, inst.ny), inst.Y, inst.r, inst.rho, T,
                      keep=tuple(range(T + 1)), Xstar=inst.Xstar)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


# power-of-two sides (radix-2 FFT), sides of other lengths (direct DFT), and
# one of each
@pytest.mark.parametrize("nx,ny,m,rho", [(16, 16, 96, 4), (32, 16, 160, 6), (8, 32, 100, 3),
                                         (20, 20, 120, 4), (12, 24, 110, 3), (16, 20, 100, 3)])
def test_fourier_one_step_parity(nx, ny, m, rho):
    inst = FourierInstance(nx=nx, ny=ny, q=12, r=2, m=m, rho=rho, seed=41, center=4)
    T = 10
    _, log = _oracle(inst, T)
    s = new_fourier_solver(inst)
    try:
        recs = one_step(Problem.fourier(inst), s, log, range(T))
    finally:
        s.close()
    check_records(recs, min_whole=T // 2)


def test_fourier_trajectory_and_init():
    inst = FourierInstance(nx=16, ny=16, q=16, r=2, m=100, rho=4, seed=42, center=4)
    T = 25
    _, log = _oracle(inst, T)
    s = new_fourier_solver(inst)
    try:
        states, eta = gpu_trajectory(s, T)
    finally:
        s.close()
    check_records(trajectory_records(Problem.fourier(inst), states, eta), min_whole=T - 2)
    rels, _ = trajectory_agreement(states, log)
    assert rels[-1] <= 1e-3, rels[-1]     # 25 iterations: both still converging


@pytest.mark.parametrize("nx,ny,m,rho,T", [(4, 256, 200, 4, 8), (2, 4096, 1000, 6, 6)])
def test_fourier_long_sides_one_step(nx, ny, m, rho, T):
    """Long power-of-two sides in the frame kernel's three-stage passes, the
    bit reversal read by the first: 256-pixel rows (a round of threads takes
    16 of them), and 4096-pixel rows (one row per round, two rounds).  One-step
    parity from the oracle."""
    inst = FourierInstance(nx=nx, ny=ny, q=12, r=2, m=m, rho=rho, seed=45 + nx,
                           mask_law="uniform", b_law="gauss")
    _, log = _oracle(inst, T)
    s = new_fourier_solver(inst)
    try:
        recs = one_step(Problem.fourier(inst), s, log, range(T))
    finally:
        s.close()
    check_records(recs, min_whole=T // 2)


def test_fourier_table1_frames_one_step():
    """The Table 1 setting (Section III): 20 x 20 frames (n = 400), uniformly
    random DFT rows, S1 values, r = 4, rho = 2 with rho_max = 5; one-step
    parity from the oracle's iterates (rho_max kept by HardThreshold)."""
    inst = FourierInstance(nx=20, ny=20, q=60, r=4, m=100, rho=2, seed=43, s_law="S1",
                           mask_law="uniform", b_law="gauss")
    T = 10
    _, log = O.run_alg1(O.FourierOperator(inst.masks, 20, 20), inst.Y, 4, 5, T,
                        keep=tuple(range(T + 1)), Xstar=inst.Xstar)
    s = new_fourier_solver(inst, rho_max=5)
    try:
        recs = one_step(Problem.fourier(inst, rho=5), s, log, range(T))
    finally:
        s.close()
    check_records(recs, min_whole=T // 2, max_excluded=0.03)


def test_fourier_128x128_m_at_0p4n():
    """m = 0.4 n on 128 x 128 frames (6554 sampled rows, the top of the
    serving mix's law): the sweep keeps the frame in shared memory and its
    m-vectors in global memory.  One-step parity from the oracle's iterates."""
    inst = FourierInstance(nx=128, ny=128, q=12, r=4, m=6554, rho=200, seed=44)
    T = 4
    _, log = _oracle(inst, T)
    s = new_fourier_solver(inst)
    try:
        recs = one_step(Problem.fourier(inst), s, log, range(T))
    finally:
        s.close()
    check_records(recs, min_whole=T // 2)
