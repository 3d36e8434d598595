"""Partition of parameter points across ranks (one process per GPU).

Every omega point is independent, so ranks need no exchange: at step s rank r
evaluates the B consecutive points starting at ((s * world + r) * B) mod K of
the K-point grid (cycling through it).  Within a step the ranks' blocks are
disjoint; over ceil(K / (world B)) steps every point is covered.
"""
import numpy as np


def step_indices(step, rank, world, B, K):
    start = ((step * world + rank) * B) % K
    return (np.arange(B) + start) % K
