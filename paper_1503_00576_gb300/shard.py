"""Counting one graph on several GPUs: the multi-GPU setup of Sec. III-E.

The paper preprocesses on one GPU, copies the edge and node arrays to the
others, and lets each device count its allotted subset of the edges.  Here
every rank (one process per GPU) runs the preprocessing itself on its own
copy of the edge array -- it is deterministic, so the arrays agree without a
copy -- and counts its share of the partner groups (tc_count_part /
tc_count_per_vertex_part).  One sum all-reduce adds the shares: the uint64
total, and in per-vertex mode the int64 counts t[] (which is why the path
has a collective at all: the shares must meet).  The degrees are complete
on every rank and need no exchange.
"""
from __future__ import annotations

from . import tc_count_part, tc_count_per_vertex_part


def count_sharded(src, dst, n: int, per_vertex: bool = False, group=None, stream=None,
                  count_part=None):
    """T (or (T, t, deg) with per_vertex) of the graph, counted as this
    rank's share and summed over the ranks of `group` (torch.distributed,
    initialised by the caller: NCCL for device tensors).  `count_part`
    replaces the share function (signature of tc_count_part, or of
    tc_count_per_vertex_part with per_vertex)."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    if per_vertex:
        share = count_part or tc_count_per_vertex_part
        T, t, deg = share(src, dst, n, rank, world, stream=stream)
        total = torch.tensor([T], dtype=torch.int64, device=t.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
        return int(total.item()), t, deg
    share = count_part or tc_count_part
    T = share(src, dst, n, rank, world, stream=stream)
    total = torch.tensor([T], dtype=torch.int64, device=src.device)
    dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    return int(total.item())
