"""Source sharding across ranks (one process per GPU).

Sources are independent in Brandes' method (paper, Section I: BC is a sum of
per-source dependencies), so a job splits into contiguous source shards, one
per rank; each rank computes its shard's partial BC vector and the partial
vectors are summed onto rank 0.  That sum is the method's only exchange step.
"""
from __future__ import annotations

import numpy as np


def shard_sources(sources, world: int, rank: int) -> np.ndarray:
    """Contiguous shard `rank` of `world` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    src = np.ascontiguousarray(sources, dtype=np.int32)
    return np.array_split(src, world)[rank]


def reduce_partial_bc(partial, dist, dst: int = 0):
    """Sums the ranks' partial BC tensors (float64) onto rank `dst` in place,
    using the process group's reduce (NCCL on GPUs, gloo on CPU)."""
    dist.reduce(partial, dst=dst, op=dist.ReduceOp.SUM)
    return partial
