"""Host logic of the multi-GPU form: one process per GPU, each an independent replica.

Propagations are independent units (batch items, stack planes, serving requests), so ranks
share no data: work is split by unit, nothing is exchanged on the data path, and the only
collectives are the timing reduction (max over ranks) and the final tally.  Works with any
torch.distributed backend (NCCL on GPUs, gloo for the CPU tests).
"""
from __future__ import annotations

import numpy as np


def item_range(n_items: int, world: int, rank: int) -> range:
    """Balanced contiguous share of n_items for `rank` (sizes differ by at most one)."""
    if not (0 <= rank < world):
        raise ValueError(f"rank {rank} outside world {world}")
    base, extra = divmod(int(n_items), int(world))
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's synthetic inputs: distinct per rank, reproducible."""
    return int(base_seed) + 1000 * int(rank)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar (e.g. elapsed ms) over the process group; identity when no
    group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput of a weak-scaling run: all ranks' units over the slowest rank's time."""
    if max_seconds <= 0:
        raise ValueError("elapsed time must be positive")
    return units_per_rank * world / max_seconds


def request_cost(n: int) -> float:
    """Relative device cost of one n x n propagation (its 80 n^2 bytes of traffic)."""
    return 80.0 * n * n


def route(sizes, world: int) -> list[list[int]]:
    """Request router for serving replicas: request i (field side sizes[i]) goes to the replica
    with the least assigned cost so far (ties to the lowest rank); arrival order is kept within
    each replica.  Deterministic, so every rank can compute the same assignment."""
    load = np.zeros(world)
    out: list[list[int]] = [[] for _ in range(world)]
    for i, n in enumerate(sizes):
        r = int(np.argmin(load))
        out[r].append(i)
        load[r] += request_cost(int(n))
    return out
