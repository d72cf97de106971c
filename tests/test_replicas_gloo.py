"""The N > 1 path (replicas on disjoint seed ranges) with two gloo ranks on CPU: shards
cover the seeds exactly once, gathered results come back in seed order and equal the
single-process results, and the timing maximum is the maximum."""
import os
import socket

import numpy as np
import pytest

from paper_2310_10750_gb300 import replicas


def test_shards_partition_the_range():
    for total in (0, 1, 7, 512, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = replicas.shard(total, world, r)
                seen.extend(range(a, b))
            assert seen == list(range(total))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, total, out):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = oracle.OracleModel(n=16, delta=2 / 16, eps=0.05, tau=5e-3, nsteps=10, ic=2)
    a, b = replicas.shard(total, world, rank)
    local = np.array([m.solve_sample(100 + s)[0] for s in range(a, b)])
    full = replicas.gather_in_order(local, total, world, rank)
    mx = replicas.max_over_ranks(float(rank + 1), world)
    out.put((rank, full.tolist(), mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_in_seed_order():
    import multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, total, port = 2, 9, _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, total, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    m = oracle.OracleModel(n=16, delta=2 / 16, eps=0.05, tau=5e-3, nsteps=10, ic=2)
    single = np.array([m.solve_sample(100 + s)[0] for s in range(total)])
    for rank, full, mx in res:
        assert np.array_equal(np.array(full), single)
        assert mx == 2.0
