"""Multi-process helpers.

The sampled-grid GPE step has no data-parallel exchange on one shell.  With
N processes (one per GPU) each rank either runs a replica of the same shell
or owns a share of a batch of independent shells; only timings and counts
are combined across ranks, never data.  torch.distributed provides the
process group (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os


def env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(weights, world, rank):
    """Indices of the items rank `rank` owns: contiguous ranges whose total
    weights (e.g. active-cell counts) are as even as a greedy split allows.
    Every item is owned by exactly one rank."""
    n = len(weights)
    total = float(sum(weights))
    bounds, acc, r = [0], 0.0, 1
    for i, w in enumerate(weights):
        acc += w
        while r < world and acc >= total * r / world and len(bounds) < world:
            bounds.append(i + 1)
            r += 1
    while len(bounds) < world:
        bounds.append(n)
    bounds.append(n)
    return list(range(bounds[rank], bounds[rank + 1]))


def _reduce(x, op):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x):
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(x):
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM)
