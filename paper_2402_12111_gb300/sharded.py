"""Path sharding over ranks (torch.distributed): one estimator over N x P paths.

Paths are independent and their Philox counters depend only on the path index,
so rank r simulates the contiguous range shard_range(paths, r, world) and the
only exchange is one all-reduce (sum) of the FP64 per-strike sums -- the
paper's reduction over paths (Sec. 6) split across devices.  The normalisation
of the combined sums runs in the library (simr_finalize_sums).
"""
from __future__ import annotations

import torch.distributed as dist

from . import api


def shard_range(paths: int, rank: int, world: int):
    """(first path, count) of `rank`: contiguous blocks, the first paths % world ranks one longer."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, rem = divmod(int(paths), int(world))
    begin = rank * base + min(rank, rem)
    return begin, base + (1 if rank < rem else 0)


def sharded_sums(model, strikes, is_put: bool, steps: int, paths: int, seed: int = 1, greeks=(),
                 rel_bump: float = 1e-4, option_index: int = 0, group=None, sums_fn=None):
    """This rank's raw sums over its shard, all-reduced (summed) over the group.

    sums_fn defaults to the library's simr_path_sums; it receives
    (model, strikes, is_put, steps, path_begin, path_count, seed=, greeks=,
    rel_bump=, option_index=) and returns a [n_strikes, n_acc] FP64 tensor.
    """
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    begin, count = shard_range(paths, rank, world)
    fn = sums_fn or api.path_sums
    s = fn(model, strikes, is_put, steps, begin, count, seed=seed, greeks=greeks, rel_bump=rel_bump,
           option_index=option_index)
    if world > 1:
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    return s


def price_greeks(model, strikes, is_put: bool, steps: int, paths: int, seed: int = 1, greeks=(),
                 rel_bump: float = 1e-4, option_index: int = 0, group=None):
    """(price, stderr, greeks) of the combined N-rank estimator, on every rank."""
    s = sharded_sums(model, strikes, is_put, steps, paths, seed, greeks, rel_bump, option_index, group)
    return api.finalize_sums(model, strikes, is_put, steps, paths, s, greeks=greeks, rel_bump=rel_bump)


__all__ = ["shard_range", "sharded_sums", "price_greeks"]
