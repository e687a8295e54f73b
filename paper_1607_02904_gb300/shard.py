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


def shard_cells(sizes, world: int, rank: int, neighbours=4.0):
    """Indices of the systems that ``rank`` evaluates: the rank's part of the
    cost-balanced partition of all systems (every rank computes the same
    partition from the same sizes, so no exchange is needed to agree on it)."""
    return partition(system_cost(sizes, neighbours), world)[rank]


def fit_step(local_step):
    """One data-parallel fitting step: ``local_step()`` evaluates this rank's
    systems and returns (loss, grad) as tensors (the loss of its systems and
    its gradient with respect to the parameter table); both are then summed
    over ranks in place, giving every rank the loss and gradient of the whole
    batch."""
    loss, grad = local_step()
    allreduce_sum(grad, loss)
    return loss, grad
