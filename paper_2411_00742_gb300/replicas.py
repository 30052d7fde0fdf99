"""Host-side helpers for running the solver on several GPUs of one node.

The 2-D grid is not split across GPUs (one grid per process, replicas only);
batches of independent instances are partitioned across ranks with no data
exchange.  Only timing needs a collective: the job time is the maximum over
ranks.  These helpers hold no solver arithmetic."""
from __future__ import annotations

import numpy as np


def shard(costs, rank: int, world: int) -> list[int]:
    """Indices of the instances rank `rank` of `world` takes: greedy
    longest-processing-time assignment on the given cost estimates, so every
    rank gets about the same work; deterministic on every rank."""
    order = np.argsort(-np.asarray(costs, dtype=np.float64), kind="stable")
    load = np.zeros(world)
    owner = np.empty(len(order), dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return [int(i) for i in np.nonzero(owner == rank)[0]]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks of the default process group (the
    value itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
