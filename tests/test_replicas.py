"""Multi-rank host logic (CPU, gloo, world size 2): batch sharding and the timing reductions
that bench.py uses with one process per GPU."""
import os
import socket

import numpy as np
import pytest

from paper_1209_1910_gb300 import inputs
from paper_1209_1910_gb300.replicas import lpt_shards, problem_cost


def test_lpt_shards_partition_and_balance():
    ns = inputs.batch_sizes()
    costs = [problem_cost(n) for n in ns]
    for world in (1, 2, 3, 8):
        shards = lpt_shards(costs, world)
        flat = sorted(q for s in shards for q in s)
        assert flat == list(range(len(ns)))  # every problem exactly once
        loads = [sum(costs[q] for q in s) for s in shards]
        # LPT: no rank exceeds the mean by more than the largest single cost
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-6
    assert lpt_shards([], 2) == [[], []]
    assert lpt_shards([5.0], 3) == [[0], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_1209_1910_gb300.replicas import lpt_shards, problem_cost, reduce_max, reduce_sum

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ns = inputs.batch_sizes(64, seed=5)
    shard = lpt_shards([problem_cost(n) for n in ns], world)[rank]
    # each rank "solves" its shard: its eigenvector count and a fake elapsed time
    mine = float(sum(ns[q] for q in shard))
    total = reduce_sum(mine, dist)
    slowest = reduce_max(1.0 + rank, dist)
    out.put((rank, shard, mine, total, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    ns = inputs.batch_sizes(64, seed=5)
    (_, s0, m0, t0, x0), (_, s1, m1, t1, x1) = res
    assert sorted(s0 + s1) == list(range(len(ns))) and not set(s0) & set(s1)
    assert t0 == t1 == m0 + m1 == float(sum(ns))
    assert x0 == x1 == 2.0
