"""Sharding the point sum over several GPUs (one process per GPU).

a_lm = sum_i w_i Y*_lm(n_i) is a sum over independent points (Eq. alm_def), so
each rank transforms a contiguous shard of every catalog and one all-reduce
(sum) of the partial a_lm and of the shot-noise matrix completes the field;
the pseudo-C_l is then computed locally.  Shards depend only on (n, rank,
world), so every rank agrees on them without communication.
"""
from __future__ import annotations


def shard_bounds(n: int, rank: int, world: int):
    """[lo, hi) of rank's contiguous share of n items (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} / world {world}")
    return n * rank // world, n * (rank + 1) // world


def shard_array(arr, rank: int, world: int):
    lo, hi = shard_bounds(arr.shape[0], rank, world)
    return arr[lo:hi]


def allreduce_sum(tensors, group=None):
    """Sum each tensor over ranks in place (complex tensors via their real view)."""
    import torch
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(torch.view_as_real(t) if t.is_complex() else t, op=dist.ReduceOp.SUM, group=group)
