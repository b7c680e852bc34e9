"""Error conventions of the C ABI on a GPU (include/lrs.h).

* Handle states CREATED -> MEASURED -> INITIALISED -> ITERATING: a call made
  in the wrong state returns LRS_ERR_STATE and changes nothing (the handle
  then runs exactly as a fresh one).
* A column whose r x r Gram G_k = (A_k U)^T (A_k U) is not positive definite
  (here A_k = 0, so A_k U has rank 0 and the least-squares step for b_k,
  Eq. bk_LS, has no unique solution) makes the call return
  LRS_ERR_NUMERICAL with that column's index in lrs_last_error().
"""
import numpy as np
import pytest

from lrsgen import GaussianInstance
from tests.gpu_helpers import gpu_available, new_solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


@pytest.mark.parametrize("engine", [1, 2, 3])
def test_out_of_order_calls_return_state_error_and_change_nothing(engine):
    from paper_2311_03824_gb300 import Solver
    from paper_2311_03824_gb300 import lrs as L
    inst = GaussianInstance(n=64, q=16, r=2, m=32, rho=2, seed=5)
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, engine=engine)
    try:
        for call in (lambda: L.lrs_init(s.h), lambda: L.lrs_iterate(s.h, 1), s.get, s.X):
            with pytest.raises(L.LrsError) as e:
                call()
            assert e.value.status == L.LRS_ERR_STATE, str(e.value)
        s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                           np.ascontiguousarray(inst.A, np.float32))
        for call in (lambda: L.lrs_iterate(s.h, 1), s.get, s.X):
            with pytest.raises(L.LrsError) as e:
                call()
            assert e.value.status == L.LRS_ERR_STATE, str(e.value)
        s.init()
        s.iterate(3)
        X = s.X()
    finally:
        s.close()
    f = new_solver(inst, engine=engine)
    try:
        f.init()
        f.iterate(3)
        X_fresh = f.X()
    finally:
        f.close()
    assert np.array_equal(X, X_fresh)


@pytest.mark.parametrize("engine", [1, 2, 3])
def test_rank_deficient_column_reports_numerical_error_with_column(engine):
    from paper_2311_03824_gb300 import lrs as L
    inst = GaussianInstance(n=64, q=16, r=2, m=32, rho=2, seed=6)
    inst.A[5] = 0.0
    inst.Y[5] = 0.0
    s = new_solver(inst, engine=engine)
    try:
        with pytest.raises(L.LrsError) as e:
            s.init()
        assert e.value.status == L.LRS_ERR_NUMERICAL, str(e.value)
        assert "column 5" in str(e.value), str(e.value)
    finally:
        s.close()


def test_expired_device_wait_returns_timeout_and_the_device_stays_usable():
    """Failure detection without a fault: the task engine's queue gets one
    ticket that nothing publishes (test_withhold), the producer that pops it
    waits 200 ms (wait_ms), sets the launch's abort flag, every other wait of
    the launch returns, and the call reports LRS_ERR_TIMEOUT.  A solver
    created afterwards runs normally."""
    import time
    from paper_2311_03824_gb300 import lrs as L
    inst = GaussianInstance(n=64, q=16, r=2, m=32, rho=2, seed=7)
    s = new_solver(inst, engine=2, wait_ms=200, test_withhold=1)
    try:
        t0 = time.time()
        with pytest.raises(L.LrsError) as e:
            s.init()
        assert e.value.status == L.LRS_ERR_TIMEOUT, str(e.value)
        assert time.time() - t0 < 30
    finally:
        s.close()
    f = new_solver(inst, engine=2)
    try:
        f.init()
        f.iterate(30)
        X = f.X()
    finally:
        f.close()
    assert np.linalg.norm(X - inst.Xstar) / np.linalg.norm(inst.Xstar) < 0.5
