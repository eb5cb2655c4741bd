"""Pin (CPU) of the fractional knapsack that the screening tests use as their oracle side.

The screening GPU tests decide which lines cannot bind with `knapsack_flow_range`: the
exact maximum and minimum of a line's flow phi . p - f_d over the generator box with the
balance sum p = D, by greedy filling in coefficient order.  Here that greedy answer is
checked against a general LP solver on random small instances (HiGHS, through
scipy.optimize.linprog), so that the screening checks rest on something other than
themselves.
"""
import numpy as np
import pytest

from test_gpu_screen import knapsack_flow_range

linprog = pytest.importorskip("scipy.optimize").linprog


@pytest.mark.parametrize("seed", range(12))
def test_knapsack_flow_range_matches_lp(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    pmin = rng.uniform(0.0, 0.5, n)
    pmax = pmin + rng.uniform(0.1, 2.0, n)
    D = float(pmin.sum() + rng.uniform(0.05, 0.95) * (pmax - pmin).sum())
    phi = rng.normal(0.0, 1.0, n)
    fd = float(rng.normal(0.0, 0.5))
    hi, lo = knapsack_flow_range(phi, pmin, pmax, D, fd)
    kw = dict(A_eq=np.ones((1, n)), b_eq=[D], bounds=list(zip(pmin, pmax)), method="highs")
    rmax = linprog(-phi, **kw)
    rmin = linprog(phi, **kw)
    assert rmax.status == 0 and rmin.status == 0
    assert abs(hi - (-rmax.fun - fd)) <= 1e-9 * (1.0 + abs(hi))
    assert abs(lo - (rmin.fun - fd)) <= 1e-9 * (1.0 + abs(lo))
    assert lo <= hi


def test_knapsack_flow_range_hand_case():
    # two generators, coefficients 1 and -1, boxes [0, 1], demand 1: the flow ranges
    # over [-1, 1] (all of the demand on either generator)
    hi, lo = knapsack_flow_range(np.array([1.0, -1.0]), np.zeros(2), np.ones(2), 1.0, 0.0)
    assert hi == 1.0 and lo == -1.0
