"""Multi-GPU host logic: images are independent, so N ranks (one process per
GPU) each run their own shard with no collective on the data path.  This
module assigns images to ranks and reduces per-rank timings; results stay
on their rank (or are gathered on the host by the caller).
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_images(pixels, world: int) -> list[np.ndarray]:
    """Greedy longest-first assignment of images (by pixel count) to `world`
    ranks; returns each rank's image indices in ascending order.  The most
    loaded rank gets at most max(pixels) more than the average."""
    pixels = np.asarray(pixels, dtype=np.int64)
    order = np.argsort(-pixels, kind="stable")
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(int(i))
        heapq.heappush(heap, (load + int(pixels[i]), r))
    return [np.array(sorted(s), dtype=np.int64) for s in out]


def rank_seeds(rank: int, images_per_rank: int) -> np.ndarray:
    """Seeds of a rank's own images in the weak-scaling benchmark."""
    return np.arange(images_per_rank, dtype=np.uint64) + np.uint64(rank * images_per_rank)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest per-rank value (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
