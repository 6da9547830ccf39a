"""Multi-process layout of independent simulations.

Simulations share nothing, so the work shards across ranks (one process per
GPU) with no collective on the data path: each rank runs its own block of
simulations.  The only cross-rank operations are host-side: a barrier and a
max-reduction of elapsed times for timing, and (for a GA generation) an
all-gather of per-simulation results (24 bytes each) so every rank can rank
the whole population.
"""
from __future__ import annotations

import os

import numpy as np


def env_rank():
    """(rank, world_size, local_rank) from the torchrun environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def shard_range(n: int, rank: int, world: int):
    """Contiguous block [lo, hi) of n items owned by `rank`; blocks differ in
    size by at most one and cover 0..n-1 exactly once."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def rank_seed_offset(rank: int, per_rank: int) -> int:
    """First replicate seed of a rank in a weak-scaling run (disjoint seed
    ranges, so no two ranks simulate the same fire)."""
    return 1 + rank * per_rank


def gather_results(results: np.ndarray, world: int):
    """All-gather a structured result array over the default process group
    (rank order); identity when world == 1."""
    if world == 1:
        return results
    import torch
    import torch.distributed as dist

    raw = torch.from_numpy(np.ascontiguousarray(results).view(np.uint8).copy())
    n = torch.tensor([raw.numel()], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n)
    mx = int(max(s.item() for s in sizes))
    pad = torch.zeros(mx, dtype=torch.uint8)
    pad[: raw.numel()] = raw
    bufs = [torch.zeros(mx, dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(bufs, pad)
    parts = [b[: int(s.item())].numpy().view(results.dtype)
             for b, s in zip(bufs, sizes)]
    return np.concatenate(parts)


def sum_over_ranks(x: int, world: int, device=None) -> int:
    """Sum of an integer count over all ranks (a collective: every rank
    calls it)."""
    if world == 1:
        return int(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([int(x)], dtype=torch.int64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sharded_results(n: int, simulate_shard, rank: int, world: int):
    """Results of n independent simulations computed by `world` ranks: rank r
    runs simulate_shard(lo, hi) on its contiguous block [lo, hi) and one
    all-gather (the only collective) returns the whole batch, in index
    order, on every rank."""
    lo, hi = shard_range(n, rank, world)
    mine = simulate_shard(lo, hi)
    if len(mine) != hi - lo:
        raise ValueError(f"rank {rank}: shard [{lo}, {hi}) returned "
                         f"{len(mine)} results")
    return gather_results(mine, world)
