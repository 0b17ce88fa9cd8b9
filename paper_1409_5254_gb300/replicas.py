"""Host-side logic of multi-GPU runs: independent work per rank, no data exchange.

The long-horizon problem does not shard, so N ranks run N independent
replicas; batches shard by instances.  Ranks exchange only timings (one
max-reduction after the timed region) -- the solve itself has no collective.
"""
from __future__ import annotations

import os

import numpy as np


def rank_info():
    """(rank, local_rank, world_size) from the torchrun environment (1 process by default)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks (x itself without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank, ms_max: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return float(np.sum(units_per_rank)) / (ms_max * 1e-3)


def partition_instances(weights, world: int):
    """Split instance indices into `world` shards of nearly equal total weight.

    Longest-processing-time greedy: instances in decreasing weight go to the
    currently lightest shard.  Every index lands in exactly one shard; each
    shard's total exceeds the mean by at most the largest single weight.
    Shards are returned sorted by index (instance order within a rank)."""
    w = np.asarray(weights, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = np.zeros(world)
    shards = [[] for _ in range(world)]
    for i in np.argsort(-w, kind="stable"):
        r = int(np.argmin(loads))
        shards[r].append(int(i))
        loads[r] += w[i]
    return [np.array(sorted(s), dtype=np.int64) for s in shards]
