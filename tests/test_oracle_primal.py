"""Pins of the oracle's primal recovery (oracle/primal.py) against hand-solved cases,
closed forms and weak duality.

Hand cases (tests/golden/hand_cases.json, solved in test_oracle_pins.py):
  two-bus, mu = 0: a uniform price gives the merit order p_bal = (1.5, 0), whose flow
    1.5 exceeds the limit 1. The proportional reference (0.75, 0.75) has flow 0.75, so
    t = (1.5 - 1) / (1.5 - 0.75) = 2/3 and p = (1, 0.5): the optimum, ub = 25.
  two-bus at its optimal duals (lambda = -10, mu_hi = 20): both units are tied, every
    balanced split has flow 1.5 - p2 <= 1, so no repair, and ub >= gamma* = 25.
  three-bus, mu = 0: merit order (2, 0) has f_01 = 4/3 > 1. The reference (1, 1) sits
    on the limit, so t = 1 and ub = 30 = gamma*.
"""
import json
import os

import numpy as np
import pytest

from oracle import dcopf, exact, primal
from paper_2406_13191_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def hand(name):
    d = json.load(open(GOLD))[name]
    net = dcopf.Net(d["n_bus"], d["line_from"], d["line_to"], d["line_b"], d["flow_max"], None,
                    d["gen_bus"], d["pmin"], d["pmax"], d["cost_lin"], None, base_mva=1.0)
    return net, np.array(d["loads"]), d


def onet(s):
    return dcopf.Net.from_dict(s.as_dict())


def test_two_bus_merit_order_repaired_to_the_optimum():
    net, loads, d = hand("two_bus")
    zero = np.zeros(net.n_line)
    for lam in (-20.0, 0.0, -5.0):
        r = primal.recover(net, loads, lam, zero, zero)
        assert r["status"] == 0
        assert abs(r["t"] - 2.0 / 3.0) < 1e-12
        assert np.allclose(r["p"], [1.0, 0.5], atol=1e-12)
        assert abs(r["ub"] - 25.0) < 1e-12
        assert r["maxviol"] <= 1e-12


def test_two_bus_at_the_optimal_duals():
    """Both units are tied at the optimal duals (up to the rounding of the prices), so
    the balanced minimiser is one of the dispatches that fill the demand between
    the tied units; every one of them has flow 1.5 - p2 <= 1 here, so no repair is
    needed, and the bound is valid but not tight (an LP's optimal duals do not
    identify its primal optimum)."""
    net, loads, d = hand("two_bus")
    r = primal.recover(net, loads, d["lambda"], np.array(d["mu_hi"]), np.array(d["mu_lo"]))
    assert r["status"] == 0 and r["t"] == 0.0
    p = r["p"]
    assert abs(p.sum() - 1.5) < 1e-12 and np.all(p >= -1e-15) and np.all(p <= 2 + 1e-15)
    assert r["ub"] == pytest.approx(10 * p[0] + 30 * p[1], rel=1e-14)
    assert r["ub"] >= d["gamma"] - 1e-12


def test_three_bus_reference_on_the_limit():
    net, loads, d = hand("three_bus")
    zero = np.zeros(net.n_line)
    r = primal.recover(net, loads, -15.0, zero, zero)
    assert r["status"] == 0
    assert abs(r["t"] - 1.0) < 1e-12
    assert np.allclose(r["p"], [1.0, 1.0], atol=1e-12)
    assert abs(r["ub"] - d["gamma"]) < 1e-12


@pytest.mark.parametrize("qp", [False, True])
def test_no_binding_lines_gives_the_economic_dispatch(qp):
    """With mu = 0 the prices are uniform, and the balance step is the economic
    dispatch: the merit order (LP) or equal incremental cost (QP), for any lambda."""
    s, loads = synth.tiny_network(21 if qp else 20, 8, 11, 6, quadratic=qp)
    d = s.as_dict()
    d["flow_max"] = np.full(s.n_line, 1e6)
    d["flow_min"] = -d["flow_max"]
    net = dcopf.Net.from_dict(d)
    D = loads.sum()
    if qp:
        def disp(lam):
            return np.clip((-lam / net.S - net.c) / (2 * net.a * net.S), net.pmin, net.pmax)
        lo, hi = -1e6, 0.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if disp(mid).sum() > D else (lo, mid)
        p = disp(0.5 * (lo + hi))
        gamma = float(np.sum(net.a * (net.S * p) ** 2 + net.c * net.S * p))
    else:
        rem, gamma = D, 0.0
        for j in np.argsort(net.c):
            take = min(rem, net.pmax[j])
            gamma += net.c[j] * net.S * take
            rem -= take
    zero = np.zeros(net.n_line)
    for lam in (-3000.0, 0.0, 750.0):
        r = primal.recover(net, loads, lam, zero, zero)
        assert r["status"] == 0 and r["t"] == 0.0
        assert abs(r["ub"] - gamma) <= 1e-9 * gamma
        assert abs(r["p"].sum() - D) <= 1e-12 * D


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_qp_at_the_dual_optimum_recovers_the_optimum(seed):
    """Strictly convex costs: the minimiser at the optimal duals is the primal optimum,
    so the recovery needs neither shift nor repair and ub = gamma*."""
    s, loads = synth.tiny_network(seed, 9, 13, 5, quadratic=True, tight=0.5)
    net = onet(s)
    r0 = exact.ipm(net, loads)
    assert r0["status"] == "optimal"
    r = primal.recover(net, loads, r0["lam"], r0["mu_hi"], r0["mu_lo"])
    assert r["status"] == 0
    assert abs(r["ub"] - r0["gamma"]) <= 1e-7 * abs(r0["gamma"])
    assert r["t"] <= 1e-6


@pytest.mark.parametrize("qp", [False, True])
def test_random_dual_points_give_feasible_upper_bounds(qp):
    """Weak duality (Remarks 1-2): whatever the dual point, the recovered dispatch is
    feasible (box, balance, limits) and costs at least gamma* (vertex enumeration for
    the LP, the interior point for the QP)."""
    rng = np.random.default_rng(7)
    for seed in range(40, 46):
        s, loads = synth.tiny_network(seed, 5, 6, 4, quadratic=qp, tight=0.5)
        net = onet(s)
        gamma = exact.vertex_enumeration(net, loads)[0] if not qp else exact.ipm(net, loads)["gamma"]
        for _ in range(5):
            lam = -rng.uniform(500, 6000)
            mh = rng.exponential(300, net.n_line) * (rng.random(net.n_line) < 0.5)
            ml = rng.exponential(300, net.n_line) * (rng.random(net.n_line) < 0.5)
            r = primal.recover(net, loads, lam, mh, ml)
            if r["status"] != 0:
                assert r["status"] == 2   # the proportional reference was infeasible
                continue
            p = r["p"]
            assert np.all(p >= net.pmin - 1e-12) and np.all(p <= net.pmax + 1e-12)
            assert abs(p.sum() - loads.sum()) <= 1e-12 * loads.sum()
            f = net.flows(net.gen_injection(p) - loads)
            assert np.all(f <= net.fmax + 1e-9) and np.all(f >= net.fmin - 1e-9)
            assert r["ub"] >= gamma - 1e-9 * abs(gamma)
            assert r["ub"] == pytest.approx(net.cost(p), rel=1e-14)


def test_statuses():
    net, loads, d = hand("two_bus")
    zero = np.zeros(net.n_line)
    assert primal.recover(net, loads * 10, -10.0, zero, zero)["status"] == 1   # D > sum pmax
    ok = np.array([0.0, 1.5])        # balanced and in the box, flow 1.5 - 1.5 = 0: feasible
    assert primal.recover(net, loads, -10.0, zero, zero, p_ref=ok)["status"] == 0
    bad = np.array([1.5, 0.0])       # flow 1.5 > 1: infeasible reference
    r = primal.recover(net, loads, -10.0, zero, zero, p_ref=bad)
    assert r["status"] == 2 and r["ub"] == np.inf
    for bad in ([0.5, 1.5 + 1e-6], [-0.5, 2.0], [2.5, -1.0]):   # unbalanced; outside the box
        assert primal.recover(net, loads, -10.0, zero, zero, p_ref=np.array(bad))["status"] == 2


def test_balance_candidate():
    """Two-bus by hand: (0.5, 0.5) totals 1 < 1.5, the room to pmax is 3, so
    phi = 1/6 and the candidate moves to (0.75, 0.75). Random candidates: the result
    stays in the box and meets the demand; a balanced candidate is left as it is."""
    net, loads, d = hand("two_bus")
    assert np.allclose(primal.balance_candidate(net, [0.5, 0.5], 1.5), [0.75, 0.75], atol=1e-15)
    assert np.allclose(primal.balance_candidate(net, [1.0, 0.5], 1.5), [1.0, 0.5], atol=1e-15)
    s, loads = synth.tiny_network(50, 9, 12, 7)
    net = onet(s)
    rng = np.random.default_rng(3)
    D = loads.sum()
    for _ in range(20):
        pc = rng.uniform(net.pmin, net.pmax)
        p = primal.balance_candidate(net, pc, D)
        assert np.all(p >= net.pmin - 1e-15) and np.all(p <= net.pmax + 1e-15)
        assert abs(p.sum() - D) <= 1e-12 * D
    assert primal.balance_candidate(net, pc, net.pmax.sum() * 1.01) is None


@pytest.mark.parametrize("qp", [False, True])
def test_mean_dispatch_candidate(qp):
    """dcopf.solve's mean_dispatch is the k^2-weighted mean of the minimisers of the
    recorded evaluations; recovered from it, the bound is feasible and above gamma*."""
    s, loads = synth.tiny_network(60 if qp else 61, 6, 8, 4, quadratic=qp, tight=0.5)
    net = onet(s)
    r = dcopf.solve(net, loads, rule="adam", alpha=500.0, beta1=0.95, max_iters=150, record=True)
    ps = [dcopf.dual_parts(net, loads, l, h, lo)[3] for (l, h, lo) in r["points"]]
    w = np.arange(1, len(ps) + 1, dtype=float) ** 2
    assert np.allclose(r["mean_dispatch"], (w[:, None] * np.array(ps)).sum(0) / w.sum(), rtol=1e-13)
    gamma = exact.vertex_enumeration(net, loads)[0] if not qp else exact.ipm(net, loads)["gamma"]
    rec = primal.recover(net, loads, r["lam"], r["mu_hi"], r["mu_lo"], p_cand=r["mean_dispatch"])
    if rec["status"] == 0:
        f = net.flows(net.gen_injection(rec["p"]) - loads)
        assert np.all(f <= net.fmax + 1e-9) and np.all(f >= net.fmin - 1e-9)
        assert abs(rec["p"].sum() - loads.sum()) <= 1e-12 * loads.sum()
        assert rec["ub"] >= gamma - 1e-9 * abs(gamma)
    else:
        assert rec["status"] == 2
