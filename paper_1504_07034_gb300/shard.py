"""Sharding of independent 1-D problems (batched shock tubes) across ranks.

The tubes of a batch never exchange data, so a batch splits across GPUs by instance with
no collective on the data path.  The work of tube b to a final time t is its lattice
updates, N_b cells times ceil(t lambda_b N_b) steps (dt = dx / lambda_b, dx = 1 / N_b),
so the cost is taken proportional to lambda_b N_b^2.  ``lpt_shards`` assigns the tubes
greedily, largest cost first, each to the currently least-loaded rank (longest
processing time first), whose makespan is at most 4/3 - 1/(3 parts) of the optimum.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def tube_costs(lengths: Sequence[int], lambdas: Sequence[float]) -> list[float]:
    """Relative work of each tube: lambda_b N_b^2."""
    return [float(lam) * float(n) * float(n) for n, lam in zip(lengths, lambdas)]


def lpt_shards(costs: Sequence[float], parts: int) -> list[list[int]]:
    """Indices of the tubes of each of `parts` shards (each list in increasing index order)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    heap = [(0.0, r) for r in range(parts)]
    shards: list[list[int]] = [[] for _ in range(parts)]
    for b in order:
        load, r = heapq.heappop(heap)
        shards[r].append(b)
        heapq.heappush(heap, (load + costs[b], r))
    return [sorted(s) for s in shards]


def shard_loads(costs: Sequence[float], shards: Sequence[Sequence[int]]) -> list[float]:
    return [sum(costs[b] for b in s) for s in shards]
