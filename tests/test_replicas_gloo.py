"""Multi-process host logic on CPU (gloo, world size 2): instance sharding
covers every instance exactly once with balanced work, and the job-time /
work reductions agree across ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2411_00742_gb300 import replicas


def test_shard_partitions_and_balances():
    rng = np.random.default_rng(0)
    costs = rng.uniform(1, 100, 4096)
    parts = [replicas.shard(costs, r, 4) for r in range(4)]
    allidx = sorted(i for p in parts for i in p)
    assert allidx == list(range(4096))
    loads = [costs[p].sum() for p in parts]
    assert max(loads) / min(loads) < 1.01


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = np.arange(1, 101, dtype=np.float64)
    mine = replicas.shard(costs, rank, world)
    t = 1.0 + rank            # per-rank "time"
    work = float(costs[mine].sum())
    q.put((rank, mine, replicas.max_over_ranks(t), replicas.sum_over_ranks(work)))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert sorted(out[0][1] + out[1][1]) == list(range(100))
    assert out[0][2] == out[1][2] == 2.0
    assert out[0][3] == out[1][3] == float(np.arange(1, 101).sum())
