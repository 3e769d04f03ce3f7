"""Host-side logic for running the solver on several GPUs of one node.

A single grid does not shard (every line step of a sweep reads its
neighbours' values of the step before), so several GPUs run independent
replicas; a batch of independent grids shards with no data exchange at all
(each rank solves its own subset).  The only collectives are the timing
ones: the max over ranks of the timed region and the sum of the work units
every rank processed.  One process per GPU, launched by torchrun; the same
functions run on CPU ranks over gloo (tests).
"""
from __future__ import annotations

import torch


def shard(sizes, rank, world):
    """Indices of the items rank `rank` of `world` solves: greedy balance by
    size (largest first, to the least-loaded rank; ties to the lower rank),
    deterministic on every rank.  The shards are disjoint and cover all."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    mine = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += sizes[i]
        mine[r].append(i)
    return sorted(mine[rank])


def _group():
    return torch.distributed.is_available() and torch.distributed.is_initialized()


def max_over_ranks(ms, device="cpu"):
    """The slowest rank's time (ms); the value itself on one process."""
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if _group() and torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device="cpu"):
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if _group() and torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_local, ms_local, device="cpu"):
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time.  Returns (units per second, max ms)."""
    ms = max_over_ranks(ms_local, device)
    units = sum_over_ranks(units_local, device)
    return units / (ms / 1e3), ms
