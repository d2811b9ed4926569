"""Data-parallel sharding of quartet work across ranks (one process per GPU).

Quartets are independent (every (ab|cd) block is its own output), so the
path shards without any exchange of data: each rank evaluates its own share
of the quartet list into its own output buffer.  The only collective is the
timing reduction (maximum of the per-rank step times).
"""
from __future__ import annotations

import numpy as np


def shard_quartets(quartets: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Rank `rank`'s share of a quartet list: every world-th quartet starting
    at `rank` (strided, so that each rank receives the same class mix)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world: {}/{}".format(rank, world))
    return np.ascontiguousarray(quartets[rank::world])


def shard_sizes(n: int, world: int) -> list:
    """Number of quartets each rank receives from shard_quartets."""
    return [(n - r + world - 1) // world for r in range(world)]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank scalar over the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
