"""The N > 1 path of bench.py on CPU: two gloo ranks (spawned processes,
rendezvous on 127.0.0.1) take the slowest rank's time, report the same
whole-job value, and solve different problems; the reference arm's other
ranks leave without work.  No GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms_local = 10.0 + 5.0 * rank          # rank 1 is the slow one
        dist.barrier()
        ms = bench.max_over_ranks(ms_local, w, "cpu")
        value = bench.whole_job_value(w, 1000, 200, ms)
        from lrsgen import GaussianInstance
        inst = GaussianInstance(n=40, q=6, r=2, m=20, rho=2, seed=bench.rank_seed(2, r))
        out[rank] = (r, w, local, ms, value, float(inst.A[0, 0, 0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time_and_solve_different_problems():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, local, ms, value, a00) in res.items():
        assert (r, w, local) == (rank, world, rank)
        assert ms == 15.0                              # max over ranks
        assert value == pytest.approx(2 * 1000 * 200 / 0.015)
    assert res[0][5] != res[1][5]                      # different seeds, different A_k


def test_single_rank_is_a_no_op():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_value(1, 1000, 200, 1000.0) == pytest.approx(200_000.0)
    assert bench.rank_seed(2, 0) == 2 and bench.rank_seed(2, 3) == 5


def test_reference_arm_other_ranks_leave_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1) or (1.0, 1.0, 1))

    class A:
        steps, warmup = 2, 3
    assert bench.run_reference(A()) == 0
    assert called == []
