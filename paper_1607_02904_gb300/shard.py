"""Sharding a batch of independent systems over ranks (one process per GPU).

The systems of a fitting batch are independent: each rank evaluates its own
subset in one batched launch and the only exchange is the sum of the
parameter-gradient vectors and of the loss over ranks. Host logic only.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition(costs, world: int):
    """Greedy longest-processing-time assignment: systems in decreasing cost,
    each to the rank with the least total so far (ties: lowest rank). Returns
    one sorted index list per rank."""
    costs = np.asarray(costs, dtype=np.float64)
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    for i in sorted(range(costs.size), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def system_cost(n_atoms, neighbours=4.0):
    """Work of one system: atoms x neighbours^2 (three-body terms per atom)."""
    return np.asarray(n_atoms, dtype=np.float64) * neighbours * neighbours


def allreduce_sum(*tensors):
    """Sums tensors over all ranks in place (gradient vector and loss)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return tensors
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors
