"""Reduced-precision storage of A_k (BF16, FP8 e4m3 hi, FP8 e4m3 hi/lo) with
defect correction, through the C ABI, against the FP64 oracle of the same
scheme (oracle/storage_forms.py: the oracle decodes the stored form itself
and runs Algorithm 1 on it with the corrected measurements) and against the
exact-operator oracle for the final error.

Bars: one-step parity (refinement every iteration) at 1e-5 with identical
supports where the oracle's margin exceeds 1e-4, over all sweep shapes; the
final iterate of a full run (initialisation, then T iterations with
refinement every 8) within 1e-5 of the final iterate of Algorithm 1 with the
exact operator in FP64, and of the scheme's own oracle.

A rounded operator can put a column's IHT on a trajectory that amplifies
rounding (the initialisation's ten sweeps from zero, with mu alternating
between two values, are the usual place): FP32 and FP64 then take such a
column through different supports although every HardThreshold margin is
large.  One-step comparisons measure this by rerunning the oracle's step
with rounding-size perturbations inside the IHT (tests/gpu_helpers.py):
supports that move are not compared, and the iterate's bar is 10 x the
perturbation's effect when that exceeds 1e-5.  Whole trajectories are not
compared iterate by iterate for these forms (a single such column makes the
paths differ while both converge to the same solution, which the final-
iterate bar checks).
"""
import numpy as np
import pytest

import oracle.storage_forms as F
from lrsgen import GaussianInstance
import oracle.altgdmin_lrs as O
from tests.gpu_helpers import (TOL, gpu_available, new_solver, one_step, oracle_run, rel,
                               step_sensitivity, x_of)
from tests.test_gpu_parity import check_one_step

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


def step_sens(inst, form, log, ts):
    """Sensitivity of each one-step comparison (refinement every iteration)."""
    At, _ = F.encode(inst.A, form)
    return step_sensitivity(O.GaussianOperator(At),
                            lambda t: F.corrected_measurements(inst.A, At, inst.Y, log.X[t]),
                            log, ts, inst.rho, inst.n)


SHAPES = [dict(engine=1, cluster=1, slab_mode=1, stages=2),
          dict(engine=1, cluster=2, slab_mode=2, stages=2),
          dict(engine=1, cluster=4, slab_mode=2, stages=2),
          dict(engine=1, cluster=8, slab_mode=1, stages=2),
          dict(engine=2), dict(engine=2, task_kib=4, inflight=3)]


@pytest.mark.parametrize("a_dtype", [1, 2, 3])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda d: "-".join(f"{k}{v}" for k, v in d.items()))
def test_one_step_all_forms_and_shapes(a_dtype, shape):
    inst = GaussianInstance(n=250, q=40, r=3, m=36, rho=3, seed=101)
    _, log = scheme_run(inst, FORMS[a_dtype], 16, 1)
    sens = step_sens(inst, FORMS[a_dtype], log, range(0, 16))
    res = one_step(inst, log, range(0, 16), sens=sens, a_dtype=a_dtype, refine_every=1, **shape)
    check_one_step(res)


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
        _, log = scheme_run(inst, FORMS[a_dtype], 6, 1)
        sens = step_sens(inst, FORMS[a_dtype], log, range(0, 6))
        res = one_step(inst, log, range(0, 6), sens=sens, a_dtype=a_dtype, refine_every=1,
                       engine=2)
        # r = 16 on m = 48 rows: the same 1e-4 bar as FP32; r = 1 on m = 24 rows
        # of which one is zero: FP32 rounding over 23 informative rows leaves
        # one-step deviations near 1e-5, so the bar is 2e-5
        edge_bar = 1e-4 if r == 16 else 2e-5
        for rr in res:
            assert rr["sup_bad"] == 0
            if rr["undecided"] == 0:
                assert rr["rel"] <= max(rr["bar"], edge_bar), rr
