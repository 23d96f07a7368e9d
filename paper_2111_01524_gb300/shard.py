"""Sharding of independent work units (grids of a batch, requests of a
stream) across ranks, one GPU per rank.

The units of the batched and served workloads are independent problems: a
grid or a request never reads another's state, so N GPUs take disjoint
subsets and exchange nothing on the data path. The only communication is
the host-side bookkeeping of the measurement (a barrier, the slowest rank's
time and the total of the units processed).

``balance`` assigns units by estimated work (cells x steps) with the
longest-processing-time rule: units in decreasing order of work, each to the
rank with the least work so far (ties to the lower rank). The assignment is
a pure function of the weights and the world size, so every rank computes
the same partition without communicating.
"""
from __future__ import annotations

import heapq

import numpy as np


def balance(weights, world):
    """Partition unit indices 0..len(weights)-1 over ``world`` ranks.

    Returns a list of ``world`` lists of unit indices, each in increasing
    order; every unit appears exactly once.
    """
    if world < 1:
        raise ValueError(f"world size must be >= 1, got {world}")
    w = np.asarray(weights, dtype=np.float64)
    if w.ndim != 1 or (w.size and (not np.all(np.isfinite(w)) or w.min() < 0)):
        raise ValueError("weights must be a 1-D array of finite non-negative numbers")
    # decreasing weight, then increasing index (stable, deterministic)
    order = sorted(range(w.size), key=lambda i: (-w[i], i))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(w[i]), r))
    return [sorted(p) for p in parts]


def loads(weights, parts):
    """Total weight of each part."""
    w = np.asarray(weights, dtype=np.float64)
    return [float(w[p].sum()) if len(p) else 0.0 for p in parts]
