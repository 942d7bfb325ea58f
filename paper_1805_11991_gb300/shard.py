"""Sharding a counting job over ranks (one process per GPU).

Members are independent, so rank r of N takes a contiguous slice of each job's
member range and counts it on its own GPU; the histograms of disjoint slices
add exactly (``hwc_hist_merge``).  The only exchange is one gather of the
sparse (tuple, multiplicity) lists at the end, done here with
``torch.distributed.all_gather_object`` on any backend.
"""
from __future__ import annotations

import numpy as np

from . import hwc


def shard_range(first: int, count: int, rank: int, world: int):
    """Contiguous slice [a, a + n) of [first, first + count) for `rank`."""
    a = first + (count * rank) // world
    b = first + (count * (rank + 1)) // world
    return a, b - a


def gather_merge(h: "hwc.Histogram", group=None) -> "hwc.Histogram":
    """All ranks' histograms of disjoint slices, added (every rank gets it)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    payload = (h.g, h.counts.tolist(), h.mult.tolist(), h.n_squarefree, h.n_total)
    dist.all_gather_object(parts, payload, group=group)
    acc = None
    for g, counts, mult, nsq, ntot in parts:
        part = hwc.Histogram(g, np.asarray(counts, np.int32).reshape(-1, g), np.asarray(mult, np.uint64),
                             nsq, ntot)
        acc = part if acc is None else hwc.hist_merge(acc, part)
    return acc


def count_sharded(g: int, q: int, fam: "hwc.Family", first: int, count: int, flags: int = 0, group=None):
    """Count this rank's slice on its GPU and return the merged histogram."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    a, n = shard_range(first, count, rank, world)
    return gather_merge(hwc.count(g, q, fam, a, n, flags), group)
