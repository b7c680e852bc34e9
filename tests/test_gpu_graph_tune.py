"""CUDA-graph replay of the steady GDmin iteration and the task-engine
autotuner, through the C ABI.

* graph replay (use_graph = 1 on a stream) gives bit-identical iterates to
  eager launches, for both sweep engines and for a low-precision form (two
  captured graphs: with and without the refinement of the measurements);
* lrs_autotune restores the iterate it starts from: a run tuned after the
  initialisation ends within 1e-5 of an untuned run and of the FP64 oracle,
  and a later handle of the same shape starts with the cached choice.
"""
import numpy as np
import pytest

from lrsgen import GaussianInstance
from tests.gpu_helpers import TOL, gpu_available, oracle_run, rel, x_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2311_03824_gb300 import build
    build.build()


def run(inst, T, **opts):
    import torch
    from paper_2311_03824_gb300 import Solver
    stream = torch.cuda.Stream()
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, stream=stream, **opts)
    try:
        s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                           np.ascontiguousarray(inst.A, np.float32))
        s.init()
        for _ in range(T):
            s.iterate(1)
        return s.get()
    finally:
        s.close()


@pytest.mark.parametrize("opts", [dict(engine=1), dict(engine=2), dict(engine=2, a_dtype=1),
                                  dict(engine=2, a_dtype=2, refine_every=3)],
                         ids=lambda d: "-".join(f"{k}{v}" for k, v in d.items()))
def test_graph_replay_is_bit_identical(opts):
    inst = GaussianInstance(n=200, q=120, r=3, m=80, rho=4, seed=21)
    eager = run(inst, 12, use_graph=0, **opts)
    graph = run(inst, 12, use_graph=1, **opts)
    for a, b in zip(eager, graph):
        assert np.array_equal(a, b)


def test_autotune_restores_state_and_caches():
    import torch
    from paper_2311_03824_gb300 import Solver
    from paper_2311_03824_gb300 import lrs as L
    inst = GaussianInstance(n=300, q=96, r=4, m=90, rho=5, seed=22)
    T = 60
    _, log = oracle_run(inst, T)
    stream = torch.cuda.Stream()
    s = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, stream=stream, engine=2)
    s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                       np.ascontiguousarray(inst.A, np.float32))
    s.init()
    before = s.get()
    rep = L.lrs_autotune(s.h, 2)
    after = s.get()
    for a, b in zip(before, after):          # the iterate is restored exactly
        assert np.array_equal(a, b)
    assert len(rep["trials"]) >= 3 and rep["chosen"]["ms"] > 0
    assert s.progress()[1] == 0
    s.iterate(T)
    X = x_of(*s.get(), inst.q)
    s.close()
    assert rel(X, log.X[-1]) <= TOL
    X0 = x_of(*run(inst, T, engine=2), inst.q)
    assert rel(X, X0) <= TOL
    # a new handle of this shape starts with the cached choice
    s2 = Solver(inst.n, inst.m, inst.q, inst.r, inst.rho, stream=stream, engine=2)
    d = L.lrs_describe(s2.h)
    s2.close()
    assert d["inflight"] == rep["chosen"]["inflight"]
