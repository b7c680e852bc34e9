"""Column-sharded solves on CPU ranks (paper_2311_03824_gb300/sharded.py):
the column split, the exchange of partial-sum blocks between two gloo ranks
(spawned processes, rendezvous on 127.0.0.1), the library's reducer callback
driven through ctypes, and the protocol's claim: the gradient of Section
II-A summed from per-rank blocks in column order equals, bit for bit, the one
summed by a single rank over the same blocks.  No GPU (the device side of the
same claim: tests/test_gpu_sharded.py)."""
import ctypes
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_03824_gb300.sharded import exchange_blocks, make_reducer, shard_columns


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("q,world,gb", [(200, 2, 16), (37, 2, 8), (37, 3, 8), (5, 3, 2),
                                        (128, 2, 64), (100, 8, 7)])
def test_shard_columns_cover_in_whole_blocks(q, world, gb):
    sh = shard_columns(q, world, gb)
    assert len(sh) == world
    assert sh[0][0] == 0 and sh[-1][1] == q
    for (a0, a1), (b0, b1) in zip(sh, sh[1:]):
        assert a1 == b0
    for k0, k1 in sh:
        assert k0 % gb == 0 and k0 <= k1
    sizes = [-(-(k1 - k0) // gb) for k0, k1 in sh]
    assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1


def test_shard_columns_needs_a_block_per_rank():
    with pytest.raises(ValueError):
        shard_columns(5, 4, 2)


def block_partials(H, Bk, k0, k1, gb):
    """Partial sums sum_k h_k b_k^T over blocks of gb columns of [k0, k1),
    each added in column order in float32."""
    out = []
    for b0 in range(k0, k1, gb):
        acc = np.zeros((H.shape[1], Bk.shape[1]), np.float32)
        for k in range(b0, min(k1, b0 + gb)):
            acc = acc + np.outer(H[k], Bk[k]).astype(np.float32)
        out.append(acc)
    return np.stack(out)


def sum_in_order(blocks):
    g = np.zeros(blocks.shape[1:], np.float32)
    for b in blocks:
        g = g + b
    return g


def gradient_terms(seed=3):
    """h_k = A_k^T (A_k (U b_k + s_k) - y_k) and b_k of an oracle iterate,
    rounded to float32 (the values the device reduction adds)."""
    import oracle.altgdmin_lrs as O
    from lrsgen import GaussianInstance
    inst = GaussianInstance(n=60, q=37, r=3, m=30, rho=2, seed=seed)
    op = O.GaussianOperator(inst.A)
    st, _, _, _ = O.init_alg1(op, inst.Y, inst.r, inst.rho)
    X = st.U @ st.B + st.S.T
    res = op.A(X.T) - np.asarray(inst.Y, np.float64)
    H = op.AH(res).astype(np.float32)            # q x n
    return H, st.B.T.astype(np.float32), O.gradient_U(op, st.U, st.B, st.S, inst.Y)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # 1. the exchange: uneven block counts, rank order kept
        rng = np.random.default_rng(100 + rank)
        mine = rng.standard_normal((3 - rank, 5, 2)).astype(np.float32)
        got = exchange_blocks(mine)
        # 2. the reducer callback as the library calls it (host pointers)
        cb, errors = make_reducer(exchange_blocks)
        cap = 6
        buf_out = (ctypes.c_float * (cap * 5 * 2))()
        m = np.ascontiguousarray(mine)
        nb_all = cb(None, m.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), m.shape[0], 5, 2,
                    buf_out, cap)
        via_cb = np.ctypeslib.as_array(buf_out).reshape(cap, 5, 2)[:max(nb_all, 0)].copy()
        # 3. the sharded gradient against one rank's
        H, Bk, _ = gradient_terms()
        gb = 8
        k0, k1 = shard_columns(H.shape[0], world, gb)[rank]
        blocks = exchange_blocks(block_partials(H, Bk, k0, k1, gb))
        out[rank] = (got, nb_all, via_cb, [repr(e) for e in errors], sum_in_order(blocks))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_and_sum_bit_for_bit():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    want = np.concatenate([np.random.default_rng(100 + r).standard_normal((3 - r, 5, 2))
                           .astype(np.float32) for r in range(world)])
    H, Bk, grad64 = gradient_terms()
    single = sum_in_order(block_partials(H, Bk, 0, H.shape[0], 8))
    for rank in range(world):
        got, nb_all, via_cb, errors, grad = res[rank]
        assert np.array_equal(got, want)
        assert errors == [] and nb_all == 5 and np.array_equal(via_cb, want)
        assert np.array_equal(grad, single)          # bit for bit
    # and the sum is the gradient of Section II-A (float32 terms)
    np.testing.assert_allclose(single, grad64, rtol=1e-5, atol=1e-5 * np.abs(grad64).max())


def test_reducer_reports_a_failed_exchange():
    def broken(mine):
        raise RuntimeError("peer gone")
    cb, errors = make_reducer(broken)
    mine = np.zeros((1, 4, 2), np.float32)
    buf = (ctypes.c_float * 8)()
    rc = cb(None, mine.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1, 4, 2, buf, 1)
    assert rc < 0 and "peer gone" in repr(errors[0])
    cb2, errors2 = make_reducer(lambda m: np.zeros((3, 4, 2), np.float32))   # over capacity
    assert cb2(None, mine.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1, 4, 2, buf, 1) < 0
    assert errors2
