"""Batches of gathers sharded over ranks (one process per GPU).

The gathers of a batch are independent problems, so the multi-GPU form of a
batch is a set of replicas: rank r takes one contiguous shard of the gather
list, builds its own ``Batch`` of that shard on its own GPU and transforms it;
the per-gather results are then concatenated on the host in the original
order. Nothing is exchanged on the data path; the only communication is the
host-side collection of the finished results.

    lo, hi = shard_bounds(weights, world)[rank]
    batch = Batch(geometries[lo:hi])
    ...                                   # transforms of the shard
    images = gather_in_order(local_images, world)   # every gather, in order
"""
from __future__ import annotations

from typing import Sequence


def shard_bounds(weights: Sequence[float] | int, world: int) -> list[tuple[int, int]]:
    """Contiguous shards [lo, hi) of n items for `world` ranks, in rank order.

    `weights` gives each item's cost (e.g. its samples Nt * Nx), or is the
    item count n (equal costs). Cut k is placed where the running cost first
    reaches k / world of the total, so every shard's cost is within one item
    of an equal split; every item lands in exactly one shard and shards may
    be empty when n < world."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = [1.0] * weights if isinstance(weights, int) else [float(v) for v in weights]
    if any(v < 0 for v in w):
        raise ValueError("weights must be non-negative")
    n = len(w)
    total = sum(w)
    cuts = [0]
    run, i = 0.0, 0
    for k in range(1, world):
        target = total * k / world
        while i < n and run + 0.5 * w[i] < target:
            run += w[i]
            i += 1
        cuts.append(max(i, cuts[-1]))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def gather_in_order(local: list, world: int, group=None) -> list:
    """Concatenate every rank's list of per-item results in rank order (rank
    0's items first): with contiguous shards from ``shard_bounds`` this is the
    original item order. Results should be host objects (numpy arrays or CPU
    tensors). With world == 1 the list is returned as is."""
    if world == 1:
        return list(local)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, list(local), group=group)
    out = []
    for p in parts:
        out.extend(p)
    return out
