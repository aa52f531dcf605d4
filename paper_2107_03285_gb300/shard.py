"""Sharding of independent design instances over ranks (one GPU per rank).

A batch of instances has no coupling: every instance is its own subtree of
the elimination forest, so ranks take disjoint subsets and need no
collective on the data path, only a final reduction of timings.  Instances
are assigned by estimated factorization cost, largest first, each to the
currently least-loaded rank (longest-processing-time greedy), which keeps
the ranks within a few percent of each other for the uneven sizes of a
batch.
"""
from __future__ import annotations

import numpy as np


def instance_costs(sides, dim=2):
    """Estimated factorization cost of square grid instances with the given
    side lengths (nodes per side): nested dissection of an n-node 2D grid
    costs O(n^{3/2}) = O(side^3) flops, a 3D cube O(n^2) = O(side^6)."""
    s = np.asarray(sides, dtype=np.float64)
    return s ** 3 if dim == 2 else s ** 6


def partition(costs, n_ranks):
    """Disjoint, deterministic assignment of instances to n_ranks ranks:
    returns a list of n_ranks sorted index arrays."""
    costs = np.asarray(costs, dtype=np.float64)
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = np.zeros(n_ranks)
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        r = int(np.argmin(load))  # first least-loaded rank on ties
        parts[r].append(i)
        load[r] += costs[i]
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def max_over_ranks(value, device=None):
    """The largest value over all ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
