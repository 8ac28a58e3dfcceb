"""Host-side sharding of walks across ranks and the merge of their accumulators.

Every (point, walk) of the method is independent (Sec. 1: the walks are trivially
parallel), so ranks never exchange data while walking.  A rank either takes a
contiguous block of points, or all points with a disjoint range of walk ids (the
Philox counter includes the walk id, so the ranks' streams never overlap).  The
only exchange is one sum of the FP64 accumulators (sum, sumsq, count) at the end.
"""
from __future__ import annotations


def point_range(rank: int, world: int, npts: int):
    """Contiguous block [start, end) of points for `rank`; blocks differ in size by at most one."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(npts, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def walk_range(rank: int, world: int, walks_per_point: int, walk_offset: int = 0):
    """(walk_offset, walks) of `rank` when every rank walks all points: disjoint walk-id ranges
    that together cover walk_offset .. walk_offset + walks_per_point - 1."""
    s, e = point_range(rank, world, walks_per_point)
    return walk_offset + s, e - s


def merge_accumulators(accum, group=None):
    """Sum (sum, sumsq, count) over the ranks of `group` in place (torch.distributed, any backend)."""
    import torch.distributed as dist
    for t in accum:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return accum
