"""Ensemble host logic on CPU: the LPT placement (paper Sec. 2.2.3, Fig.
balance) pinned against Graham's bound for longest-processing-time-first on
brute-forced optima, its ordering rules, the cost estimate's monotonicity,
and the seeded C4 recipe."""
import itertools
import math

import numpy as np
import pytest

from inputs.workloads import c4_ensemble
from paper_2512_12629_gb300 import cube2


def _makespan(costs, bins, m):
    load = np.zeros(m)
    for c, b in zip(costs, bins):
        load[b] += c
    return load.max()


@pytest.mark.parametrize("seed", range(12))
def test_lpt_within_grahams_bound_of_the_optimum(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(3, 9)), int(rng.integers(2, 4))
    costs = rng.uniform(0.1, 10.0, n)
    bins = cube2.lpt_partition(costs, m)
    assert bins.min() >= 0 and bins.max() < m
    opt = min(_makespan(costs, a, m) for a in itertools.product(range(m), repeat=n))
    # LPT makespan <= (4/3 - 1/(3m)) OPT  (Graham 1969)
    assert _makespan(costs, bins, m) <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt * (1 + 1e-12)


def test_lpt_order_and_ties():
    # the m largest go to bins 0..m-1 in decreasing order; equal costs keep index order
    assert list(cube2.lpt_partition([1.0, 5.0, 3.0, 4.0], 3)) == [2, 0, 2, 1]
    assert list(cube2.lpt_partition([2.0] * 7, 3)) == [0, 1, 2, 0, 1, 2, 0]
    assert list(cube2.lpt_partition([], 4)) == []


@pytest.mark.parametrize("costs,bins", [([1.0, -1.0], 2), ([1.0, float("nan")], 2), ([1.0], 0),
                                        ([1.0, float("inf")], 2)])
def test_lpt_rejects_bad_input(costs, bins):
    with pytest.raises(cube2.Cube2Error):
        cube2.lpt_partition(costs, bins)


def test_cost_estimate_grows_with_the_box():
    ws = c4_ensemble(n_boxes=4, sizes=(32, 48, 64, 96))
    by_np = {}
    for w in c4_ensemble(n_boxes=64):
        by_np[w.n_p] = cube2.config_cost(cube2.make_config(w))
    ks = sorted(by_np)
    assert all(by_np[a] < by_np[b] for a, b in zip(ks, ks[1:]))
    assert len(ws) == 4


def test_c4_recipe():
    e = c4_ensemble()
    assert len(e) == 64
    assert {w.n_p for w in e} <= {32, 48, 64, 96}
    assert all(0.7 <= w.sigma8 <= 0.9 for w in e)
    assert [w.seed for w in e] == list(range(100, 164))
    assert e == c4_ensemble()
    for w in e:
        n = w.levels[0].n_mesh
        assert n == 2 * w.n_p and w.box == 2.0 * w.n_p and w.n_ios == w.n_p
        m = n
        while m % 2 == 0:
            m //= 2
        while m % 3 == 0:
            m //= 3
        assert m == 1                                  # 2^a 3^b mesh
        # PP range (2 mesh cells) equals the IOS cell
        assert math.isclose(w.levels[0].beta * w.box / n, w.box / w.n_ios)
