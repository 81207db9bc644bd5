"""Sharding of independent cells across ranks (one process per GPU).

Cells of the chemistry step never exchange data, so ranks need no collective on the data path:
each rank advances its own contiguous range of cells.  For a shared field the ranges balance
the expected work, taken as the previous step's per-cell attempt counts (accepted + rejected
sub-steps, plus one), the load-balancing use of the integrator's counters.
"""
from __future__ import annotations

import numpy as np


def partition_by_weight(weights, world):
    """Contiguous ranges [start, end) for each rank whose summed weights are as equal as a
    contiguous split allows (boundaries at the cumulative-weight quantiles)."""
    w = np.asarray(weights, np.float64)
    if w.ndim != 1 or world < 1:
        raise ValueError("weights must be 1-D and world >= 1")
    n = w.size
    if n == 0:
        return [(0, 0)] * world
    cum = np.concatenate([[0.0], np.cumsum(np.maximum(w, 0.0))])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        b = int(np.searchsorted(cum, total * r / world, side="left"))
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def shard(n, rank, world, weights=None):
    """This rank's range of n cells (equal counts, or balanced weights when given)."""
    if weights is None:
        weights = np.ones(n)
    return partition_by_weight(weights, world)[rank]
