"""Partition of work across ranks (one process per GPU).

Every omega point is independent, so ranks need no exchange:
- one dataset: at step s rank r evaluates the B consecutive points starting
  at ((s * world + r) * B) mod K of the K-point grid (cycling through it);
  within a step the ranks' blocks are disjoint, and over ceil(K / (world B))
  steps every point is covered;
- datasets of uneven size: whole datasets go to ranks, balanced by their cost
  (points x n^3, the factorisation's share): largest first, each to the rank
  with the least cost so far.
"""
import numpy as np


def step_indices(step, rank, world, B, K):
    start = ((step * world + rank) * B) % K
    return (np.arange(B) + start) % K


def balance_by_cost(costs, world):
    """Rank of every item: greedy largest-first assignment of the items to the
    rank with the smallest total cost so far (ties to the lower rank)."""
    costs = np.asarray(costs, dtype=float)
    load = np.zeros(world)
    owner = np.empty(len(costs), dtype=np.int64)
    for i in np.argsort(-costs, kind="stable"):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return owner
