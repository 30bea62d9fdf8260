"""Assignment of independent systems to GPUs for batched evaluation.

Independent systems need no exchange between GPUs: each rank evaluates its
own share in one graph launch.  Shares are balanced by the
longest-processing-time rule on a cost estimate per system (N log N: the
near field and spreading grow with N, the FFTs with N log N).
"""
from __future__ import annotations

import heapq
import math


def system_cost(n: int) -> float:
    return n * math.log2(max(n, 2))


def shard_systems(sizes, world: int):
    """Indices of the systems each of `world` ranks evaluates: systems taken
    in decreasing cost, each to the rank with the least cost so far (ties to
    the lower rank).  Every system goes to exactly one rank; each list is
    in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-system_cost(sizes[i]), i))
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + system_cost(sizes[i]), r))
    return [sorted(s) for s in shards]
