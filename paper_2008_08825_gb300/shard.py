"""Sharding of a batch of independent BSE instances over ranks (one GPU each).

A batch of independent problems (the batched workload: many instances of
uneven size n_i) splits across ranks without any exchange on the data path:
each rank solves its own instances with one persistent launch, and only the
small per-instance results travel, to rank 0, on the host.

The cost of one instance is proportional to n_i^3 (every step of Alg. 2 and
Alg. 3 is O(n^3) except the element-wise ones), so the instances are dealt by
the longest-processing-time greedy rule on n_i^3: in decreasing cost order,
each goes to the rank with the smallest load so far (lowest rank on ties).
The rule is deterministic, so every rank computes the same partition from the
sizes alone, with no communication.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_by_cost(sizes, world: int) -> list[list[int]]:
    """Indices of the instances of each rank (each list ascending).

    sizes: the n_i of the batch; world: number of ranks (>= 1).
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = np.asarray(sizes, dtype=np.int64)
    cost = sizes.astype(np.float64) ** 3
    order = sorted(range(len(sizes)), key=lambda i: (-cost[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + cost[i], r))
    return [sorted(p) for p in parts]


def loads(sizes, parts) -> list[float]:
    """Sum of n_i^3 per rank."""
    sizes = np.asarray(sizes, dtype=np.float64)
    return [float(np.sum(sizes[p] ** 3)) for p in parts]


def gather_to_rank0(local: dict, dist=None):
    """Gather per-rank {instance index: result} dictionaries on rank 0 (host
    objects over the default process group; every rank must call it).

    Returns the merged dictionary on rank 0 and None elsewhere; with no
    process group (dist None or not initialised) returns ``local``.
    """
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return dict(local)
    world = dist.get_world_size()
    out = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(local, out, dst=0)
    if dist.get_rank() != 0:
        return None
    merged: dict = {}
    for part in out:
        overlap = merged.keys() & part.keys()
        if overlap:
            raise RuntimeError(f"instances solved on two ranks: {sorted(overlap)[:5]}")
        merged.update(part)
    return merged
