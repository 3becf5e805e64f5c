"""Multi-process host logic on CPU (world size 2, gloo): sharding of independent
instances and the max-over-ranks timing that bench.py reports."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2304_02327_gb300 import parallel, workloads as wl


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, sizes, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [parallel.instance_cost(n) for n in sizes]
        mine = parallel.shard_for_rank(costs, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        # each rank "times" its shard: cost-proportional fake seconds
        t = sum(costs[i] for i in mine) / 1e9 + 0.001 * rank
        tmax = parallel.max_over_ranks(t)
        out[rank] = (gathered, t, tmax)
    finally:
        dist.destroy_process_group()


def test_lpt_partition_properties():
    costs = [5, 3, 3, 2, 2, 2, 1]
    bins = parallel.lpt_partition(costs, 3)
    assert sorted(i for b in bins for i in b) == list(range(len(costs)))
    loads = [sum(costs[i] for i in b) for b in bins]
    assert max(loads) - min(loads) <= max(costs)
    assert parallel.lpt_partition(costs, 3) == bins            # deterministic
    with pytest.raises(ValueError):
        parallel.lpt_partition(costs, 0)


def test_two_rank_sharding_and_max_time():
    probs = wl.batched_allen_cahn(count=64, seed=4)
    sizes = [p.n[0] for p in probs]
    world = 2
    port = free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, sizes, out), nprocs=world, join=True,
                       start_method="spawn")
    g0, t0, m0 = out[0]
    g1, t1, m1 = out[1]
    assert g0 == g1                                   # every rank sees the same partition
    shards = g0
    assert sorted(i for s in shards for i in s) == list(range(len(sizes)))   # exact cover
    costs = [parallel.instance_cost(n) for n in sizes]
    loads = [sum(costs[i] for i in s) for s in shards]
    assert max(loads) <= sum(loads) / world + max(costs)                     # LPT bound
    assert m0 == m1 == max(t0, t1)                                           # max over ranks
    assert parallel.job_throughput([1.0, 1.0], max(t0, t1)) == 2.0 / max(t0, t1)
