"""Host-side sharding of independent instances across ranks (one GPU each).

Instances are independent (each fit touches only its own y), so multi-GPU
runs split the batch with no data-path collective.  Ranks get balanced total
cost by longest-processing-time assignment: instances in descending cost,
each to the rank with the least work so far.  The cost of a fit is taken as
that of one model evaluation's recursion: N log2(N)^2 for the superfast
Schur recursion (N >= 64, Sec. III-E), N^2 for the Levinson recursion below.
"""
from __future__ import annotations

import heapq
import math

SUPERFAST_MIN_N = 64  # the library's default switch from Levinson to the superfast recursion


def fit_cost(n: int) -> float:
    """Relative cost of fitting an instance of n samples."""
    n = int(n)
    if n >= SUPERFAST_MIN_N:
        return n * math.log2(n) ** 2
    return float(n) ** 2


def balanced_shards(sizes, world: int) -> list[list[int]]:
    """Indices of `sizes` (instance lengths N) per rank, balancing the summed
    fit_cost.  Every index appears exactly once; each rank's list is
    ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-fit_cost(sizes[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + fit_cost(sizes[i]), r))
    return [sorted(x) for x in out]


def rank_shard(sizes, world: int, rank: int) -> list[int]:
    return balanced_shards(sizes, world)[rank]
