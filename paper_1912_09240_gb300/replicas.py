"""Host logic for running the hot path on several GPUs of one node.

The method has no data-path exchange that one GB300 cannot hold: every
workload fits one device, so ranks are independent replicas (weak scaling)
and independent problems of a batch are split across ranks with no
collective.  Only the timing uses the process group: a barrier on both sides
of the timed region and the maximum of the per-rank times.

Ranks draw distinct random numbers: rank r keys its Philox stream with
problem id r (the problem field of the counter), so replicas are
statistically independent ensembles.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return ws, rank, local


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(work: list[float], rank: int, world: int) -> list[int]:
    """Indices of the items rank `rank` owns when items of the given work are
    dealt to `world` ranks largest first, each to the least-loaded rank (ties
    to the lowest rank).  Deterministic, so every rank computes the same
    partition without communicating; the shards are disjoint and cover all
    items."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    load = [0.0] * world
    owner = [0] * len(work)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += work[i]
    return [i for i in range(len(work)) if owner[i] == rank]
