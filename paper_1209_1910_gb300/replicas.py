"""Host-side helpers for running the library on several GPUs of one node, one process per GPU.

The method has no exchange step between independent problems, so several GPUs are used as
replicas: a single problem is solved by every rank on its own copy (weak scaling), and a batch of
independent problems is split into per-rank shards with no collective on the data path.  The
only collectives are the timing reductions (the maximum of the ranks' elapsed times, sums of
counts) made outside the timed work.
"""
from __future__ import annotations

import os

import numpy as np


def lpt_shards(costs, world: int):
    """Split problems with the given costs over `world` ranks by the longest-processing-time rule
    (problems in decreasing cost, each to the currently least loaded rank; ties to the lowest
    rank and the lower problem index).  Returns a list of `world` sorted index lists."""
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda q: (-costs[q], q))
    load = [0.0] * world
    shards = [[] for _ in range(world)]
    for q in order:
        r = min(range(world), key=lambda i: (load[i], i))
        shards[r].append(q)
        load[r] += float(costs[q])
    return [sorted(s) for s in shards]


def problem_cost(n: int) -> float:
    """Work estimate of one problem of order n for sharding: the LU factors and the first sweep
    grow as n^2 per problem; clusters add up to n^3 but are unknown before the plan, so n^2.5 is
    used as a middle estimate."""
    return float(n) ** 2.5


def env_rank():
    """(rank, world, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value: float, dist, device=None) -> float:
    """Maximum of a host float over the ranks of the default process group."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist, device=None) -> float:
    """Sum of a host float over the ranks of the default process group."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
