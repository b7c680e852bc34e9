"""Reduced-precision storage of A_k (BF16, FP8 e4m3 hi, FP8 e4m3 hi/lo) with
defect correction, through the C ABI, against the FP64 oracle of the same
scheme (oracle/storage_forms.py: the oracle decodes the stored form itself
and runs Algorithm 1 on it with the corrected measurements) and against the
exact-operator oracle for the final error.

Bars: one-step parity (refinement every iteration) as in the FP32 tests
(tests/gpu_helpers.py): from the scheme oracle's iterate t, one GPU
iteration against the probed FP64 oracle step on the decoded operator with
the corrected measurements of X_t - supports identical and b_k, s_k within
1e-5 on the decidable columns, the whole X within 1e-5 where every column is
decidable; over all sweep shapes, and over the rank widths 8, 10 and 12
whose W products run as round-robin tasks (m = 150 rows: two W row blocks of
128 and 22 rows).  The final iterate of a full run (initialisation, then T
iterations with refinement every 8) is within 1e-5 of the final iterate of
Algorithm 1 with the exact operator in FP64, and of the scheme's own oracle.

A rounded operator can put a column's initialisation on a trajectory that
amplifies rounding (the ten sweeps from zero, with mu alternating between
two values); whole trajectories are therefore not compared iterate by
iterate for these forms, only their final iterates, which both converge to
the same solution.
"""
import numpy as np
import pytest

import oracle.storage_forms as F
from lrsgen import GaussianInstance
from tests.gpu_helpers import (TOL, Problem, check_records, gpu_available, new_solver, one_step,
                               oracle_run, rel, x_of)

pytestmark = pytest.mark.gpu

FORMS = {1: "bf16", 2: "fp8_hi", 3: "fp8_hilo"}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


def scheme_run(inst, form, T, refine_every):
    At, _ = F.encode(inst.A, form)
    return F.run_defect_corrected(inst.A, At, inst.Y, inst.r, inst.rho, T, refine_every,
                                  Xstar=inst.Xstar, keep=tuple(range(T + 1)))


def form_one_step(inst, a_dtype, T, min_whole, **shape):
    """One-step parity of a stored form, refinement before every iteration."""
    form = FORMS[a_dtype]
    At, _ = F.encode(inst.A, form)
    _, log = scheme_run(inst, form, T, 1)
    P = Problem.gaussian(inst, A=At)
    s = new_solver(inst, a_dtype=a_dtype, refine_every=1, **shape)
    try:
        recs = one_step(P, s, log, range(T),
                        y_of_t=lambda t: F.corrected_measurements(inst.A, At, inst.Y, log.X[t]))
    finally:
        s.close()
    return check_records(recs, min_whole)


SHAPES = [dict(engine=1, cluster=1, slab_mode=1, stages=2),
          dict(engine=1, cluster=2, slab_mode=2, stages=2),
          dict(engine=1, cluster=4, slab_mode=2, stages=2),
          dict(engine=1, cluster=8, slab_mode=1, stages=2),
          dict(engine=2), dict(engine=2, task_kib=4, inflight=3)]


@pytest.mark.parametrize("a_dtype", [1, 2, 3])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda d: "-".join(f"{k}{v}" for k, v in d.items()))
def test_one_step_all_forms_and_shapes(a_dtype, shape):
    inst = GaussianInstance(n=250, q=40, r=3, m=36, rho=3, seed=101)
    form_one_step(inst, a_dtype, 16, min_whole=12, **shape)


@pytest.mark.parametrize("a_dtype", [1, 2, 3])
@pytest.mark.parametrize("r", [8, 10, 12])
def test_one_step_wide_ranks_round_robin_w(r, a_dtype):
    """Rank widths 8-12: the task engine's W products run as round-robin
    tasks (a lane owns whole rows; FP8 hi sums raw codes and scales each row
    once).  m = 150 gives a ragged second W row block; n = 300 a ragged last
    tile."""
    inst = GaussianInstance(n=300, q=24, r=r, m=150, rho=5, seed=400 + r)
    form_one_step(inst, a_dtype, 8, min_whole=6, engine=2)
    form_one_step(inst, a_dtype, 4, min_whole=3, engine=2, task_kib=16, inflight=5)


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("a_dtype", [1, 2, 3])
def test_final_error(a_dtype, engine):
    """n=200, q=200, r=3, m=80, rho=4, T=150, refinement every 8 iterations:
    the stored form converges to the exact-operator FP64 solution."""
    inst = GaussianInstance(n=200, q=200, r=3, m=80, rho=4, seed=1)
    T = 150
    _, log = scheme_run(inst, FORMS[a_dtype], T, 8)
    _, exact = oracle_run(inst, T)
    assert rel(log.X[-1], exact.X[-1]) < 1e-7        # the oracles agree
    s = new_solver(inst, a_dtype=a_dtype, refine_every=8, engine=engine)
    try:
        s.init()
        s.iterate(T)
        X = x_of(*s.get(), inst.q)
    finally:
        s.close()
    assert rel(X, exact.X[-1]) <= TOL
    assert rel(X, log.X[-1]) <= TOL


@pytest.mark.parametrize("a_dtype", [1, 2, 3])
def test_zero_rows_and_rank_edges(a_dtype):
    """r = 1 and r = 16, rho = 0, and an all-zero row in every A_k (row scale 1)."""
    for r, rho, m in [(1, 2, 24), (16, 0, 48)]:
        inst = GaussianInstance(n=70, q=30, r=r, m=m, rho=rho, seed=300 + r)
        inst.A[:, 0, :] = 0.0
        inst.Y[:, 0] = 0.0
        form_one_step(inst, a_dtype, 6, min_whole=4, engine=2)
