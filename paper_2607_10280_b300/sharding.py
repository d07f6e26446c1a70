"""Splitting a batch of images over independent ranks (one process per GPU).

Every image is independent from encoding to the linear layer, so ranks never
exchange data while they compute: each takes a contiguous range of images whose
estimated cost (L * n * D^3, D the largest bond the image reaches) is balanced
across ranks.  The only collective is an optional gather of the results to one
rank at the end.
"""
from __future__ import annotations

import numpy as np


def image_cost(p: int, L: int, chi: int) -> float:
    n = p * p
    D = min(chi, 2 ** max(L, 0), 2 ** (n // 2))
    return float(max(L, 1) * n * max(D, 1) ** 3)


def shard_ranges(costs, world: int) -> list:
    """Contiguous [start, end) ranges, one per rank, with balanced summed cost.

    Rank r takes the images whose cost prefix sum falls in [r/world, (r+1)/world)
    of the total (each image goes where its cost midpoint lands), so every image is
    assigned exactly once and the ranges tile 0..len(costs)."""
    costs = np.asarray(costs, dtype=np.float64)
    n = len(costs)
    if world < 1:
        raise ValueError("world must be >= 1")
    total = costs.sum()
    if n == 0 or total <= 0:
        edges = np.linspace(0, n, world + 1).round().astype(int)
    else:
        mid = (np.cumsum(costs) - 0.5 * costs) / total          # in (0, 1)
        owner = np.minimum((mid * world).astype(int), world - 1)
        edges = [0]
        for r in range(world):
            edges.append(int(np.searchsorted(owner, r, side="right")))
        edges[-1] = n
    return [(int(edges[r]), int(edges[r + 1])) for r in range(world)]


def gather_to_root(local: np.ndarray, group=None):
    """Gather each rank's result array (first axis = images) to rank 0, in rank order.
    Returns the concatenation on rank 0 and None elsewhere."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    t = torch.from_numpy(np.ascontiguousarray(local))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([t.shape[0]], dtype=torch.int64), group=group)
    maxn = int(max(s.item() for s in sizes))
    pad = torch.zeros((maxn,) + tuple(t.shape[1:]), dtype=t.dtype)
    pad[:t.shape[0]] = t
    bufs = [torch.zeros_like(pad) for _ in range(world)] if rank == 0 else None
    dist.gather(pad, bufs, dst=0, group=group)
    if rank != 0:
        return None
    return np.concatenate([b[:int(s.item())].numpy() for b, s in zip(bufs, sizes)])
