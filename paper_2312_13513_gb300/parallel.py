"""Work across ranks (one process per GPU).

* Chemistry: cells of the chemistry step never exchange data, so ranks need no collective on the
  data path: each rank advances its own contiguous range of cells.  For a shared field the ranges
  balance the expected work, taken as the previous step's per-cell attempt counts (accepted +
  rejected sub-steps, plus one), the load-balancing use of the integrator's counters.
* Surrogate training is data-parallel: every rank holds the same network, computes the gradients
  of its equal share of each global batch, and one all-reduce (sum) of the flat gradient buffer,
  scaled by 1 / ranks, gives every rank the gradient of the mean loss over the global batch
  before the identical Adam step.  The flat layout is the library's (chem_mlp_grad_pack): layer by
  layer, dW_l [out x in] row-major, then db_l [out].
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


def batch_share(global_batch_idx, rank, world):
    """This rank's equal, contiguous share of a global batch (its size must divide by world)."""
    n = len(global_batch_idx)
    if world < 1 or n % world:
        raise ValueError(f"global batch {n} does not split into {world} equal shares")
    b = n // world
    return global_batch_idx[rank * b:(rank + 1) * b]


def flatten_grads(dW, db):
    """The flat gradient layout of chem_mlp_grad_pack, for host arrays: dW_l row-major, then db_l."""
    parts = []
    for w, b in zip(dW, db):
        parts.append(np.asarray(w).reshape(-1))
        parts.append(np.asarray(b).reshape(-1))
    return np.concatenate(parts)


def unflatten_grads(flat, shapes):
    """Inverse of flatten_grads; shapes = [(out, in), ...] per layer."""
    dW, db, o = [], [], 0
    for (r, c) in shapes:
        dW.append(np.asarray(flat[o:o + r * c]).reshape(r, c)); o += r * c
        db.append(np.asarray(flat[o:o + r])); o += r
    if o != len(flat):
        raise ValueError("flat gradient length does not match the layer shapes")
    return dW, db


def allreduce_sum_(flat, group=None):
    """Sum a flat tensor over the ranks of group in place (one collective: NCCL for CUDA
    tensors, gloo for CPU tensors).  Returns the number of ranks, 1 without torch.distributed."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return 1
    world = dist.get_world_size(group)
    if world > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    return world


def rebalance(local_weights, start, n_total, group=None):
    """Balanced contiguous ranges for the next step of a shared field of n_total cells, from the
    per-cell weights (attempt counts + 1) each rank measured on its current range [start, start +
    len(local_weights)): one all-reduce (sum) assembles the field's weights on every rank (the
    ranges tile the field, so every cell has exactly one contributor), then every rank takes its
    quantile range.  local_weights is a torch tensor on the process group's device (CUDA for NCCL,
    CPU for gloo).  Returns (start, end) of this rank; without torch.distributed, (0, n_total)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return 0, n_total
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    full = torch.zeros(n_total, dtype=torch.float64, device=local_weights.device)
    full[start:start + local_weights.numel()] = local_weights.to(torch.float64)
    if world > 1:
        dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)
    return shard(n_total, rank, world, full.cpu().numpy())
