"""Sharding of independent tubes by instance (paper_1504_07034_gb300.shard), on the CPU.

Longest-processing-time-first must assign every tube exactly once, be deterministic,
and keep the largest shard within Graham's bound 4/3 - 1/(3m) of the optimal makespan,
which brute force gives on small instances.
"""
import itertools

import numpy as np
import pytest

import workloads as W
from paper_1504_07034_gb300.shard import lpt_shards, shard_loads, tube_costs


def _optimum(costs, parts):
    best = float("inf")
    for assign in itertools.product(range(parts), repeat=len(costs)):
        loads = [0.0] * parts
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("parts", [2, 3])
def test_lpt_within_graham_bound_of_brute_force(seed, parts):
    rng = np.random.default_rng(seed)
    costs = list(rng.uniform(1.0, 100.0, size=8))
    shards = lpt_shards(costs, parts)
    assert sorted(b for s in shards for b in s) == list(range(len(costs)))
    lpt = max(shard_loads(costs, shards))
    assert lpt <= (4.0 / 3.0 - 1.0 / (3 * parts)) * _optimum(costs, parts) + 1e-9


def test_tube_batch_shards_cover_the_batch_and_balance():
    tb = W.batched_tubes(seed=0, count=512)
    costs = tube_costs(tb.lengths, tb.lam)
    # the cost model is the tube's lattice updates up to the rounding of its step count
    updates = tb.lengths * tb.steps
    assert np.allclose(np.array(costs) * tb.t_final, updates, rtol=0.02)
    for parts in (1, 2, 4, 8):
        shards = lpt_shards(costs, parts)
        assert sorted(b for s in shards for b in s) == list(range(512))
        assert shards == lpt_shards(costs, parts)                   # deterministic
        loads = shard_loads(costs, shards)
        assert max(loads) <= sum(loads) / parts + max(costs)          # greedy list-scheduling bound
        sub = tb.subset(shards[0])
        assert sub.total_updates == int(updates[shards[0]].sum())
