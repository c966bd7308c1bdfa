"""Sharding of one fit over several processes (one model per GPU).

Events and normalisation points are independent units of the likelihood
(the unbinned likelihood of the Introduction is a product over events; I of
Eq. 5 is a sum over points), so each
rank holds a contiguous range of both and, per evaluation, exchanges one block
of partial sums (Model.eval_partials: 6 + 2P doubles).  Every rank gathers all
blocks in rank order and combines them in native code
(amp4d_combine_partials), so every rank gets the same NLL and gradient bits.
"""
from __future__ import annotations

import numpy as np


def shard_range(n, rank, world):
    """Contiguous [lo, hi) of n units for rank in 0 .. world-1; the first n % world
    ranks take one unit more, so sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments n=%r rank=%r world=%r" % (n, rank, world))
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_partials(part, group=None):
    """All-gather this rank's partial block over torch.distributed; returns the
    (world, width) float64 array in rank order.  Works on gloo (CPU tensors) and
    on NCCL (the block is moved to the current CUDA device for the exchange)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.as_tensor(np.ascontiguousarray(part, dtype=np.float64), device=dev)
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t, group=group)
    return np.stack([b.cpu().numpy() for b in bufs])


def combine_gathered(parts):
    """(nll, gradient or None) of the union of the shards whose blocks are the rows
    of parts, in rank order."""
    from paper_2007_14931_gb300 import combine_partials
    nll, grad, _ = combine_partials(parts)
    return nll, grad


def sharded_eval(model, params, grad=True, group=None, stream=None):
    """One evaluation of a sharded fit: this rank's partials, the all-gather, and
    the rank-ordered combination.  Returns (nll, gradient or None)."""
    part = model.eval_partials(params, grad=grad, stream=stream)
    return combine_gathered(gather_partials(part, group))
