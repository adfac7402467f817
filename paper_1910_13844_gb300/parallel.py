"""Multi-process use of the LS model: views are independent given f (eq. prob), so they shard.

* ``shard_views`` splits Q views into contiguous, balanced ranges, one per rank.
* ``allreduce_`` sums a tensor over ranks (the gradient of eq. prob is a sum over views).
* ``data_grad_sharded`` computes this rank's share of the data term and its gradient with the
  CUDA library, then all-reduces loss and gradient: the one collective of the path.

Forward solves need no exchange at all; the bench runs independent replicas (weak scaling).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_views(n_views: int, world: int, rank: int) -> range:
    """Contiguous range of views for `rank`; sizes differ by at most one, lower ranks take the extra."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(n_views, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def allreduce_(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum over the ranks of `group` (no-op without an initialised process group)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def data_grad_sharded(prob, f: torch.Tensor, group=None, data_grad=None):
    """(loss, gradient) of the data term over all views, each rank solving its own shard.

    ``data_grad(prob, f, views) -> (loss, grad)`` evaluates the term over a list of views; the
    default is the CUDA library's (``recon.data_grad``)."""
    if data_grad is None:
        from .recon import data_grad

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    views = list(shard_views(prob.kvec.shape[0], world, rank))
    if views:
        loss, g = data_grad(prob, f, views)
    else:
        loss, g = 0.0, torch.zeros_like(f)
    lt = torch.tensor([loss], dtype=torch.float64, device=g.device)
    allreduce_(g, group)
    allreduce_(lt, group)
    return float(lt.item()), g


def gather_views(x: np.ndarray, world: int) -> list:
    """Helper for tests and tools: the per-rank slices of a per-view array."""
    return [x[list(shard_views(len(x), world, r))] for r in range(world)]
