"""Sharding a batch of independent meshes over ranks (one GPU per rank).

Meshes of a batch are independent units, so a batch splits across ranks with
no exchange in the data path: each rank adapts its share (pm_adapt_batch on
its own GPU) and only the per-mesh results come back to rank 0.  A single
mesh is not split (that would need a halo exchange between partitions); it
runs as replicas.
"""
from __future__ import annotations

import heapq


def partition(sizes, nranks):
    """Greedy longest-processing-time split: meshes in descending size go to
    the rank with the least work so far.  Returns one list of mesh indices
    per rank (each ascending); deterministic (ties to the lower index/rank)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    heap = [(0, r) for r in range(nranks)]
    out = [[] for _ in range(nranks)]
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    return [sorted(x) for x in out]


def gather_results(local, rank, world, group=None):
    """Collect {mesh index: result} dicts from every rank on rank 0 (host
    objects through torch.distributed); other ranks get None."""
    import torch.distributed as dist

    if world == 1:
        return dict(local)
    objs = [None] * world if rank == 0 else None
    dist.gather_object(dict(local), objs, dst=0, group=group)
    if rank != 0:
        return None
    merged = {}
    for o in objs:
        merged.update(o)
    return merged


def adapt_sharded(items, sizes, rank, world, adapt, group=None):
    """Adapt this rank's share of `items` (split by `sizes` with partition)
    through adapt(index, item) -> result, then gather every rank's
    {index: result} on rank 0 (None on the other ranks).  The data path has
    no exchange: each rank's meshes are adapted where they live."""
    parts = partition(sizes, world)
    local = {i: adapt(i, items[i]) for i in parts[rank]}
    return gather_results(local, rank, world, group)
