"""Host-side logic of the batch: the longest-processing-time-first plan
(nrs_batch_plan, no device needed), checked against its definition and
against Graham's bound for LPT, makespan <= (4/3 - 1/(3K)) x optimum, with
the optimum found by brute force on small instances."""

import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def N():
    from paper_2001_06468_gb300 import nrs
    return nrs


def test_plan_follows_its_definition(N):
    cost = [5.0, 3.0, 8.0, 1.0, 1.0, 9.0]
    chain, order = N.batch_plan(cost, 2)
    # decreasing cost, ties in index order
    assert list(order) == [5, 2, 0, 1, 3, 4]
    # greedy: each problem to the least-loaded chain, ties to the lower chain
    assert list(chain) == [1, 0, 1, 0, 0, 0]


def test_single_chain_and_more_chains_than_problems(N):
    chain, order = N.batch_plan([2.0, 7.0, 7.0], 1)
    assert list(chain) == [0, 0, 0] and list(order) == [1, 2, 0]
    chain, _ = N.batch_plan([2.0, 7.0, 3.0], 5)
    assert sorted(chain) == [0, 1, 2]


@pytest.mark.parametrize("seed", range(6))
def test_makespan_within_grahams_bound(N, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n, K = 7, 3
    cost = rng.uniform(1.0, 10.0, size=n)
    chain, _ = N.batch_plan(cost, K)
    makespan = max(cost[chain == k].sum() for k in range(K))
    best = min(max(sum(cost[i] for i in range(n) if a[i] == k) for k in range(K))
               for a in itertools.product(range(K), repeat=n))
    assert makespan <= (4.0 / 3.0 - 1.0 / (3 * K)) * best + 1e-12


def test_plan_rejects_bad_arguments(N):
    with pytest.raises(N.NrsError):
        N.batch_plan([], 2)
    with pytest.raises(N.NrsError):
        N.batch_plan([1.0], 0)
