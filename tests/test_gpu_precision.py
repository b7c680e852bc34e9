"""Reduced-precision storage of A_k (BF16, FP8 e4m3 hi, FP8 e4m3 hi/lo) with
defect correction, through the C ABI, against the FP64 oracle of the same
scheme (oracle/storage_forms.py: the oracle decodes the stored form itself
and runs Algorithm 1 on it with the corrected measurements) and against the
exact-operator oracle for the final error.

Bars: one-step parity (refinement every iteration) at 1e-5 with identical
supports where the oracle's margin exceeds 1e-4, over all sweep shapes;
trajectory parity against the scheme's oracle; final iterate within 1e-5 of
the exact-operator oracle's final iterate.
"""
import numpy as np
import pytest

import oracle.storage_forms as F
from lrsgen import GaussianInstance
from tests.gpu_helpers import TOL, gpu_available, one_step, oracle_run, rel, trajectory
from tests.test_gpu_parity import check_one_step, check_trajectory

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


@pytest.mark.parametrize("a_dtype", [1, 2, 3])
@pytest.mark.parametrize("cluster,slab_mode", [(1, 1), (2, 2), (4, 2), (8, 1)])
def test_one_step_all_forms_and_shapes(a_dtype, cluster, slab_mode):
    inst = GaussianInstance(n=250, q=40, r=3, m=36, rho=3, seed=101)
    _, log = scheme_run(inst, FORMS[a_dtype], 16, 1)
    res = one_step(inst, log, range(0, 16), a_dtype=a_dtype, refine_every=1, cluster=cluster,
                   slab_mode=slab_mode, stages=2)
    check_one_step(res)


@pytest.mark.parametrize("a_dtype", [1, 2, 3])
def test_trajectory_and_final_error(a_dtype):
    """n=200, q=200, r=3, m=80, rho=4, refinement every 8 iterations."""
    inst = GaussianInstance(n=200, q=200, r=3, m=80, rho=4, seed=1)
    T = 150
    _, log = scheme_run(inst, FORMS[a_dtype], T, 8)
    res, eta = trajectory(inst, T, log, a_dtype=a_dtype, refine_every=8)
    check_trajectory(res, eta, log)
    # against the exact operator: same final iterate as Algorithm 1 in FP64
    _, exact = oracle_run(inst, T)
    assert rel(log.X[-1], exact.X[-1]) < 1e-7
    from tests.gpu_helpers import new_solver, x_of
    s = new_solver(inst, a_dtype=a_dtype, refine_every=8)
    try:
        s.init()
        s.iterate(T)
        X = x_of(*s.get(), inst.q)
    finally:
        s.close()
    assert rel(X, exact.X[-1]) <= TOL


@pytest.mark.parametrize("a_dtype", [1, 2, 3])
def test_zero_rows_and_rank_edges(a_dtype):
    """r = 1 and r = 16, rho = 0, and an all-zero row in every A_k (row scale 1)."""
    for r, rho, m in [(1, 2, 24), (16, 0, 48)]:
        inst = GaussianInstance(n=70, q=30, r=r, m=m, rho=rho, seed=300 + r)
        inst.A[:, 0, :] = 0.0
        inst.Y[:, 0] = 0.0
        _, log = scheme_run(inst, FORMS[a_dtype], 6, 1)
        res = one_step(inst, log, range(0, 6), a_dtype=a_dtype, refine_every=1)
        for rr in res:
            assert rr["sup_bad"] == 0
            if rr["undecided"] == 0:
                assert rr["rel"] <= TOL, rr
