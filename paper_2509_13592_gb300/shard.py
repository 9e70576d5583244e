"""Splitting a batch of independent instances over ranks (one GPU per rank).

Instances share nothing, so there is no collective on the data path: each rank
solves its own slice.  The only collective is the max over ranks of a timing.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple


def instance_cost(L1: int, L2: int) -> float:
    """Relative cost of one iteration on an L1 x L2 grid (FFT2 + IFFT2 ~ L log L)."""
    L = L1 * L2
    return L * math.log2(L)


def partition(shapes: Sequence[Tuple[int, int]], world: int) -> List[List[int]]:
    """Assign instance indices to `world` ranks so that the summed cost per rank is
    balanced (longest-processing-time greedy); every index appears exactly once and
    each rank's list is in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(shapes)), key=lambda i: (-instance_cost(*shapes[i]), i))
    loads = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += instance_cost(*shapes[i])
    return [sorted(p) for p in parts]


def contiguous_range(n_per_rank: int, rank: int) -> range:
    """Weak scaling with a fixed per-rank batch: rank r owns instances [r n, (r + 1) n)."""
    return range(rank * n_per_rank, (rank + 1) * n_per_rank)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a host float over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
