"""Column-sharded solve on the GPU (Section II-E): two shards of one problem,
each a handle with its own columns, driven by two host threads that exchange
the n x r partial sums through the library's reducer callback (a host
barrier: the shards' kernels never wait on one another).  After the
initialisation and every iteration, U, B_k and S_k of the shards equal, bit
for bit, those of one handle over all columns with the same grad_block."""
import threading

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


class ThreadExchange:
    """All shards' blocks in rank order, among threads of one process."""

    def __init__(self, world):
        self.slots = [None] * world
        self.barrier = threading.Barrier(world, timeout=120)

    def for_rank(self, rank):
        def exchange(mine):
            self.slots[rank] = mine
            self.barrier.wait()
            out = np.concatenate(self.slots)
            self.barrier.wait()
            return out
        return exchange


def run_shards(inst, world, gb, T, **opts):
    from paper_2311_03824_gb300.sharded import ShardedSolver, shard_columns
    ranges = shard_columns(inst.q, world, gb)
    ex = ThreadExchange(world)
    results, errors = [None] * world, [None] * world

    def work(rank):
        k0, k1 = ranges[rank]
        s = None
        try:
            s = ShardedSolver(inst.n, inst.m, inst.q, inst.r, inst.rho, k0, k1, gb,
                              exchange=ex.for_rank(rank), **opts)
            s.set_measurements(np.ascontiguousarray(inst.Y[k0:k1], np.float32),
                               np.ascontiguousarray(inst.A[k0:k1], np.float32))
            s.init()
            states = [s.get()]
            for _ in range(T):
                s.iterate(1)
                states.append(s.get())
            results[rank] = states
        except BaseException as e:
            errors[rank] = (e, s.reduce_errors if s else None)
            ex.barrier.abort()
        finally:
            if s:
                s.close()

    th = [threading.Thread(target=work, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert errors == [None] * world, errors
    return ranges, results


@pytest.mark.parametrize("engine", [1, 2, 3])
def test_two_shards_equal_one_handle_bit_for_bit(engine):
    inst = GaussianInstance(n=200, q=200, r=3, m=80, rho=4, seed=1)
    gb, T = 16, 12
    opts = dict(engine=engine, grid=64)
    ranges, shards = run_shards(inst, 2, gb, T, **opts)
    one = new_solver(inst, grad_block=gb, **opts)
    try:
        one.init()
        whole = [one.get()]
        for _ in range(T):
            one.iterate(1)
            whole.append(one.get())
    finally:
        one.close()
    for t in range(T + 1):
        U, B, Si, Sv = whole[t]
        for (k0, k1), states in zip(ranges, shards):
            Us, Bs, Sis, Svs = states[t]
            assert np.array_equal(Us, U), t
            assert np.array_equal(Bs, B[:, k0:k1]), t
            assert np.array_equal(Sis, Si[k0:k1]) and np.array_equal(Svs, Sv[k0:k1]), t


def test_shard_handle_rejects_graphs_and_missing_block():
    from paper_2311_03824_gb300 import lrs as L
    from paper_2311_03824_gb300.sharded import make_reducer
    cb, _ = make_reducer(lambda m: m)
    with pytest.raises(L.LrsError) as e:
        L.lrs_create(64, 32, 16, 2, 2, L.LRS_OP_GAUSSIAN,
                     L.make_options(reduce=cb, reduce_cap=4, grad_block=0))
    assert e.value.status == L.LRS_ERR_ARG
    with pytest.raises(L.LrsError) as e:
        L.lrs_create(64, 32, 16, 2, 2, L.LRS_OP_GAUSSIAN,
                     L.make_options(reduce=cb, reduce_cap=4, grad_block=4, use_graph=1))
    assert e.value.status == L.LRS_ERR_ARG


def test_failed_exchange_fails_the_call():
    from paper_2311_03824_gb300 import lrs as L
    from paper_2311_03824_gb300.sharded import ShardedSolver
    inst = GaussianInstance(n=64, q=16, r=2, m=32, rho=2, seed=5)

    def broken(mine):
        raise RuntimeError("peer gone")

    s = ShardedSolver(inst.n, inst.m, inst.q, inst.r, inst.rho, 0, inst.q, 4, exchange=broken)
    try:
        s.set_measurements(np.ascontiguousarray(inst.Y, np.float32),
                           np.ascontiguousarray(inst.A, np.float32))
        with pytest.raises(L.LrsError) as e:
            s.init()
        assert e.value.status == L.LRS_ERR_ARG
        assert "peer gone" in repr(s.reduce_errors[0])
    finally:
        s.close()
