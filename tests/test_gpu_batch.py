"""Several problems in one persistent launch (lrs_iterate_batch): uneven
Gaussian problems whose columns share one task-engine work table per sweep
end, bit for bit, where each handle ends when iterated alone."""
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


def _run(insts, T, batched, **opts):
    from paper_2311_03824_gb300 import lrs as L
    ss = [new_solver(inst, engine=2, **opts) for inst in insts]
    try:
        for s in ss:
            s.init()
        if batched:
            L.lrs_iterate_batch([s.h for s in ss], T)
        else:
            for s in ss:
                s.iterate(T)
        return [s.get() for s in ss], [s.progress() for s in ss]
    finally:
        for s in ss:
            s.close()


@pytest.mark.parametrize("a_dtype", [0, 1, 2])
def test_uneven_problems_in_one_launch_match_alone(a_dtype):
    # rank width class 3; different n, m, q, rho (and so different task plans,
    # pieces and shared-memory needs); a ragged tile in every problem
    insts = [GaussianInstance(n=200, q=120, r=3, m=80, rho=4, seed=61),
             GaussianInstance(n=330, q=64, r=3, m=150, rho=6, seed=62),
             GaussianInstance(n=150, q=200, r=3, m=60, rho=0, seed=63)]
    T = 12
    opts = dict(a_dtype=a_dtype) if a_dtype else {}
    alone, pa = _run(insts, T, False, **opts)
    batch, pb = _run(insts, T, True, **opts)
    for a, b, x, y in zip(alone, batch, pa, pb):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
        assert x == y                      # eta and t


def test_batch_rejects_mixed_rank_widths_and_repeats():
    from paper_2311_03824_gb300 import lrs as L
    a = new_solver(GaussianInstance(n=100, q=20, r=3, m=40, rho=2, seed=64), engine=2)
    b = new_solver(GaussianInstance(n=100, q=20, r=5, m=40, rho=2, seed=65), engine=2)
    try:
        a.init()
        b.init()
        with pytest.raises(L.LrsError) as e:
            L.lrs_iterate_batch([a.h, b.h], 1)
        assert e.value.status == L.LRS_ERR_UNSUPPORTED
        with pytest.raises(L.LrsError) as e:
            L.lrs_iterate_batch([a.h, a.h], 1)
        assert e.value.status == L.LRS_ERR_ARG
    finally:
        a.close()
        b.close()
