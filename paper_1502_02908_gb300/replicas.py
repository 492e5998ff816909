"""Replicas across GPUs.

Replicates (and batch instances) are independent and share only the read-only
event schedule, so several GPUs run disjoint replicate ranges with no exchange on
the data path; each GPU draws its replicates' own Philox streams
(``replicate_base``), so the union of the ranges is identical to one GPU running
all of them.  The one collective is the final gather of the gradient-moment
sums to every rank in rank order (deterministic: the library then adds them in
that order, as it adds one GPU's replicate chunks).
"""
from __future__ import annotations

import numpy as np


def shard(R: int, world: int, rank: int):
    """Contiguous replicate range [r0, r1) of `rank` among `world` ranks."""
    base, extra = divmod(R, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def combine(parts):
    """Adds per-rank moment sums in rank order."""
    out = np.zeros_like(parts[0])
    for p in parts:
        out = out + p
    return out


def allreduce_moments(moments: np.ndarray, group=None):
    """Gathers every rank's moment sums and adds them in rank order (torch.distributed;
    gloo or nccl).  Returns the combined sums on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.as_tensor(np.ascontiguousarray(moments, np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    return combine([p.cpu().numpy() for p in parts])


def allgather_rows(rows: np.ndarray, group=None):
    """Gathers every rank's moment rows [n_rows, F, 42] (the same shape on every
    rank) and concatenates them in rank order (torch.distributed; gloo or nccl)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.as_tensor(np.ascontiguousarray(rows, np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    return np.concatenate([p.cpu().numpy() for p in parts])
