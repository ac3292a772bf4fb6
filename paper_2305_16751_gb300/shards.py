"""A forward split over the ranks of a process group (one GPU per rank).

Every rank runs `domagg_forward_shard` for its own shard of the flat map
(the point phase is repeated on every rank; the records are split by node),
the ranks exchange their partial outputs with one all-gather -- float32 sums
as float-float pairs, so the exchange adds no rounding -- and every rank
joins them with F in `domagg_combine`.  This is the one exchange step of the
method's distributed reading (Sec. 6); nothing else crosses GPUs.
"""
from __future__ import annotations


def gather(t, group=None):
    """All-gather of one tensor over the process group: the list of every
    rank's tensor, in rank order."""
    import torch
    import torch.distributed as dist
    bufs = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(bufs, t.contiguous(), group=group)
    return bufs


def forward_distributed(D, Q, w, op: str, group=None):
    """forward(D, Q, w, op) computed by all ranks of the group together: this
    rank's shard, the exchange, the join.  Every rank returns the whole
    result."""
    import torch.distributed as dist

    from . import domagg
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    out, lo = domagg.forward_shard(D, Q, w, op, rank, world)
    parts = gather(out, group)
    los = gather(lo, group) if lo is not None else None
    return domagg.combine(parts, los, op, None if op == "count" else w.dtype)
