"""Column-sharded solves (Section II-E, communication complexity; Section I-B,
the federated setting): every process holds a contiguous range of the q
columns (its A_k and y_k never leave it) and only n x r partial sums travel,
once per column reduction (each subspace-iteration step of the
initialisation, each gradient).

The library does the arithmetic (include/lrs.h, lrs_reducer): it hands the
shard's partial sums, one n x r block per `grad_block` columns, to a
reducer and adds every shard's blocks in column order on the device, so the
result is bit for bit that of one handle over all columns with the same
grad_block.  This module supplies the column split and the exchange of the
blocks through torch.distributed (all_gather in rank order, rank order =
column order).
"""
from __future__ import annotations

import ctypes
from typing import Callable, List, Optional, Tuple

import numpy as np

from . import lrs as L


def shard_columns(q: int, world: int, grad_block: int) -> List[Tuple[int, int]]:
    """Column range [k0, k1) of every rank: whole blocks of grad_block columns
    (only the last may be short), spread as evenly as the blocks allow, in
    rank order; at least one block per rank."""
    if q < 1 or world < 1 or grad_block < 1:
        raise ValueError("need q, world, grad_block >= 1")
    nb = -(-q // grad_block)
    if nb < world:
        raise ValueError(f"{nb} blocks of {grad_block} columns for {world} ranks: "
                         "every rank needs a block")
    base, extra = divmod(nb, world)
    out, b = [], 0
    for rank in range(world):
        cnt = base + (1 if rank < extra else 0)
        out.append((min(q, b * grad_block), min(q, (b + cnt) * grad_block)))
        b += cnt
    return out


def exchange_blocks(mine: np.ndarray, group=None) -> np.ndarray:
    """Every rank's partial blocks (nb_rank, n, w) concatenated in rank order:
    block counts first, then one all_gather padded to the largest count
    (CUDA tensors for an NCCL group, host tensors otherwise)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(np.ascontiguousarray(mine, np.float32)).to(dev)
    nb = torch.tensor([t.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(nb) for _ in range(world)]
    dist.all_gather(counts, nb, group=group)
    counts = [int(c.item()) for c in counts]
    pad = torch.zeros((max(counts),) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
    pad[:t.shape[0]] = t
    bufs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    return np.concatenate([b[:c].cpu().numpy() for b, c in zip(bufs, counts)])


def make_reducer(exchange: Callable[[np.ndarray], np.ndarray]):
    """An lrs_reducer that passes the shard's blocks to exchange() and writes
    what it returns (every shard's blocks in column order).  Returns the C
    function and a list that collects the exception of a failed exchange
    (the library call then fails with LRS_ERR_ARG)."""
    errors: List[BaseException] = []

    def reducer(ctx, mine, nb, n, w, out, cap):
        try:
            a = np.ctypeslib.as_array(mine, shape=(nb, n, w)).copy()
            allb = np.asarray(exchange(a), np.float32)
            if allb.ndim != 3 or allb.shape[1:] != (n, w) or not 1 <= allb.shape[0] <= cap:
                raise ValueError(f"exchange returned shape {allb.shape}, capacity {cap}")
            np.ctypeslib.as_array(out, shape=(cap, n, w))[:allb.shape[0]] = allb
            return int(allb.shape[0])
        except BaseException as ex:   # reported through the library's status
            errors.append(ex)
            return -1

    return L.LRS_REDUCER(reducer), errors


class ShardedSolver(L.Solver):
    """The shard [k0, k1) of a q-column Gaussian problem: A (q_local, m, n),
    Y (q_local, m) of its own columns.  exchange: callable (nb, n, w) ->
    (nb_all, n, w), by default exchange_blocks over the default process
    group.  k0 must be a multiple of grad_block (see shard_columns)."""

    def __init__(self, n, m, q, r, rho, k0, k1, grad_block,
                 exchange: Optional[Callable] = None, **opts):
        if k0 % grad_block or not 0 <= k0 < k1 <= q:
            raise ValueError("shard [k0, k1) must start at a multiple of grad_block")
        self.k0, self.k1, self.q_total = k0, k1, q
        self._reduce, self.reduce_errors = make_reducer(exchange or exchange_blocks)
        cap = -(-q // grad_block)
        super().__init__(n, m, k1 - k0, r, rho, grad_block=grad_block, reduce=self._reduce,
                         reduce_cap=cap, **opts)
