"""Stream partitioning across GPUs (replicas, no collective on the data path).

Streams are independent (each text chunk has its own model state, Sec. 3.11),
so a multi-GPU run gives every GPU a disjoint subset of streams and a full
weight replica.  Streams go to GPUs greedily, longest first, each to the GPU
with the fewest tokens so far (ties: lowest rank), which keeps the per-GPU
token counts within one stream length of each other.
"""
from __future__ import annotations

import heapq


def partition_streams(lengths, world: int):
    """Return, per rank, the list of stream indices it codes."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(lengths)), key=lambda j: (-int(lengths[j]), j))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for j in order:
        load, r = heapq.heappop(heap)
        parts[r].append(j)
        heapq.heappush(heap, (load + int(lengths[j]), r))
    return parts
