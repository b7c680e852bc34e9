"""CUDA solver (through the C ABI) against the FP64 oracle.

Bars (float32 arithmetic against float64):
  * one-step parity: from the oracle's iterate t, one GPU iteration matches
    the oracle's iterate t+1 to ||dX||_F / ||X||_F <= 1e-5 with identical
    supports, at every iterate whose HardThreshold decisions FP32 can resolve
    (oracle margin > 1e-4);
  * trajectory parity: a full GPU run matches the oracle at every iterate up
    to the first sub-resolution decision, supports identical on decidable
    columns throughout, and the final iterate matches within 1e-5;
  * U orthonormal to float32 precision, S indices ascending, eta equal.
"""
import numpy as np
import pytest

from lrsgen import GaussianInstance
from tests.gpu_helpers import (MARGIN_FP32, TOL, gpu_available, one_step, oracle_run,
                               trajectory)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


def check_trajectory(res, eta_gpu, log, tol=TOL, final_tol=TOL):
    for r in res:
        if r["undecided"] == 0:
            assert r["rel"] <= max(tol, r.get("bar", tol)), ("iterate", r["t"], r["rel"])
        assert r["sup_bad"] == 0, ("support mismatch on decidable columns", r)
        assert r["ortho"] < 1e-5
        assert r["ascending"]
    assert res[-1]["rel"] <= final_tol, ("final iterate", res[-1]["rel"])
    if log.eta is not None:
        assert abs(eta_gpu - log.eta) <= 1e-4 * log.eta


def check_one_step(res, tol=TOL):
    n_checked = 0
    for r in res:
        assert r["sup_bad"] == 0, r
        if r["undecided"] == 0:
            assert r["rel"] <= max(tol, r.get("bar", tol)), r
            n_checked += 1
    assert n_checked >= len(res) // 2, "too few iterates with resolvable decisions"


# Sweep engines and their launch shapes: engine 1 = one thread-block cluster
# per column (cluster size, slab resident or streamed); engine 2 = the
# persistent task engine (bytes per task, columns in flight).
SHAPES = [dict(engine=1, cluster=1, slab_mode=1), dict(engine=1, cluster=1, slab_mode=2),
          dict(engine=1, cluster=2, slab_mode=1), dict(engine=1, cluster=2, slab_mode=2),
          dict(engine=1, cluster=4, slab_mode=2), dict(engine=1, cluster=8, slab_mode=2),
          dict(engine=2), dict(engine=2, task_kib=4, inflight=3),
          dict(engine=2, task_kib=16, inflight=1), dict(engine=2, task_kib=1024)]
ENGINES = [1, 2]


def shape_id(d):
    return "-".join(f"{k}{v}" for k, v in d.items())


@pytest.mark.parametrize("shape", SHAPES, ids=shape_id)
def test_one_step_ragged_all_shapes(shape):
    # n = 250: slabs of 32-column tiles with a ragged last tile and slab
    inst = GaussianInstance(n=250, q=40, r=3, m=36, rho=3, seed=101)
    _, log = oracle_run(inst, 20)
    opts = dict(shape)
    if opts.get("engine") == 1:
        opts.setdefault("stages", 2)
    res = one_step(inst, log, range(0, 20), **opts)
    check_one_step(res)


@pytest.mark.parametrize("shape", [dict(engine=2, task_kib=8, inflight=5), dict(engine=2)],
                         ids=shape_id)
def test_one_step_tall_columns_task_engine(shape):
    """m = 300: several W row blocks and A^T row pieces per tile."""
    inst = GaussianInstance(n=140, q=24, r=4, m=300, rho=5, seed=102)
    _, log = oracle_run(inst, 8)
    res = one_step(inst, log, range(0, 8), **shape)
    check_one_step(res)


@pytest.mark.parametrize("engine", ENGINES)
def test_trajectory_config0_full(engine):
    """n=200, q=200, r=3, m=80, rho=4, 300 iterations, every iterate."""
    inst = GaussianInstance(n=200, q=200, r=3, m=80, rho=4, seed=1)
    _, log = oracle_run(inst, 300)
    res, eta = trajectory(inst, 300, log, engine=engine)
    check_trajectory(res, eta, log)
    assert log.err[-1] < 1e-6


@pytest.mark.parametrize("engine", ENGINES)
def test_one_step_config0_every_iterate(engine):
    inst = GaussianInstance(n=200, q=200, r=3, m=80, rho=4, seed=1)
    _, log = oracle_run(inst, 60)
    res = one_step(inst, log, range(0, 60), engine=engine)
    check_one_step(res)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("r,rho,m", [(1, 1, 20), (5, 0, 30), (8, 6, 40), (16, 2, 48)])
def test_edge_ranks_and_sparsity(r, rho, m, engine):
    inst = GaussianInstance(n=70, q=30, r=r, m=m, rho=rho, seed=200 + r)
    _, log = oracle_run(inst, 12)
    res = one_step(inst, log, range(0, 12), engine=engine, cluster=1)
    check_one_step(res, tol=1e-4 if r == 16 else TOL)


@pytest.mark.parametrize("engine", ENGINES)
def test_single_column_and_rho_equals_n(engine):
    inst = GaussianInstance(n=24, q=1, r=1, m=20, rho=24, seed=300)
    _, log = oracle_run(inst, 5)
    res = one_step(inst, log, range(0, 5), engine=engine)
    check_one_step(res, tol=1e-4)


@pytest.mark.parametrize("engine", ENGINES)
def test_init_matches_oracle_subspace_and_supports(engine):
    import oracle.altgdmin_lrs as O
    from tests.gpu_helpers import new_solver
    inst = GaussianInstance(n=200, q=200, r=3, m=80, rho=4, seed=1)
    st, L0, sv, margin = O.init_alg1(O.GaussianOperator(inst.A), inst.Y, 3, 4)
    s = new_solver(inst, engine=engine)
    s.init()
    U, B, S_idx, S_val = s.get()
    s.close()
    cosines = np.linalg.svd(U.T.astype(np.float64) @ st.U, compute_uv=False)
    assert np.max(np.abs(1 - cosines)) < 1e-6, cosines  # same subspace (FP32 L0, FP32 U)
    dec = margin > MARGIN_FP32
    assert np.all(np.sort(S_idx[dec], 1) == st.S_idx[dec])
