"""Host-side logic for running the path on several GPUs, one process per GPU.

The single-tensor integrator has no data-parallel split without an exchange
step (the last mode needs every fibre of the tensor), so several GPUs run
independent replicas; batches of independent problems (uneven 2D instances)
are sharded across ranks with no collective on the data path.  Only the timing
reduction (max over ranks) uses torch.distributed.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def lpt_partition(costs: Sequence[float], parts: int) -> List[List[int]]:
    """Longest-processing-time-first assignment of items to `parts` bins.

    Items are taken in decreasing cost order (ties by index) and each goes to the
    currently lightest bin (ties by bin index): a deterministic 4/3-approximation
    of the balanced partition, the same on every rank.
    """
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, b) for b in range(parts)]
    bins: List[List[int]] = [[] for _ in range(parts)]
    for i in order:
        load, b = heapq.heappop(heap)
        bins[b].append(i)
        heapq.heappush(heap, (load + float(costs[i]), b))
    return [sorted(b) for b in bins]


def shard_for_rank(costs: Sequence[float], rank: int, world: int) -> List[int]:
    """Indices of the items rank `rank` of `world` processes owns."""
    return lpt_partition(costs, world)[rank]


def instance_cost(n: int, d: int = 2) -> float:
    """Relative cost of one Tucker step of a d-dimensional n^d instance (2 d n^(d+1))."""
    return 2.0 * d * float(n) ** (d + 1)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (identity if
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: Sequence[float], seconds: float) -> float:
    """Whole-job throughput: units processed by all ranks over the max-over-ranks time."""
    return float(sum(units_per_rank)) / seconds
