"""Host-side sharding of independent instances across ranks (one GPU each).

Instances are independent (each fit touches only its own y), so multi-GPU
runs split the batch with no data-path collective.  The cost of a fit grows
like N^2 (the Levinson recursion, once per evaluation), so ranks get
balanced total N^2 by longest-processing-time assignment: instances in
descending cost, each to the rank with the least work so far.
"""
from __future__ import annotations

import heapq


def balanced_shards(sizes, world: int) -> list[list[int]]:
    """Indices of `sizes` (instance lengths N) per rank, balancing sum N^2.
    Every index appears exactly once; each rank's list is ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 2, i))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]) ** 2, r))
    return [sorted(x) for x in out]


def rank_shard(sizes, world: int, rank: int) -> list[int]:
    return balanced_shards(sizes, world)[rank]
