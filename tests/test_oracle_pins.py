"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Hand-solved cases (tests/golden/hand_cases.json):
  two-bus: gen 1 at the slack bus (10 $/p.u.h, pmax 2), gen 2 at bus 1 (30, pmax 2),
    load 1.5 at bus 1, one line limited to 1.  f = 1.5 - p2, so p = (1, 0.5) and
    gamma* = 25.  lambda = -10, mu_hi = 20 give bus prices (-10, -30) and
    g = 0 + 45 - 20 = 25.
  three-bus triangle, equal susceptances: an injection at bus 1 splits 2/3 over the
    direct line and 1/3 over the two-line path.  Load 2 at bus 1, cheap gen at the
    slack (10), dear gen at bus 2 (20), line 0->1 limited to 1: f_01 = 4/3 - p_B/3,
    so p = (1, 1), gamma* = 30, lambda = -10, mu_hi(0->1) = 30.
"""
import json
import os

import numpy as np
import pytest

from oracle import dcopf, exact
from paper_2406_13191_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def hand(name):
    d = json.load(open(GOLD))[name]
    net = dcopf.Net(d["n_bus"], d["line_from"], d["line_to"], d["line_b"], d["flow_max"], None,
                    d["gen_bus"], d["pmin"], d["pmax"], d["cost_lin"], None, base_mva=1.0)
    return net, np.array(d["loads"]), d


def onet(net: synth.Network):
    return dcopf.Net.from_dict(net.as_dict())


@pytest.mark.parametrize("name", ["two_bus", "three_bus"])
def test_hand_cases(name):
    net, loads, d = hand(name)
    r = exact.ipm(net, loads)
    assert r["status"] == "optimal"
    assert abs(r["gamma"] - d["gamma"]) < 1e-8
    assert np.allclose(r["p"], d["p"], atol=1e-7)
    gv, _ = exact.vertex_enumeration(net, loads)
    assert abs(gv - d["gamma"]) < 1e-9
    lam, mh, ml = d["lambda"], np.array(d["mu_hi"]), np.array(d["mu_lo"])
    for fn in (dcopf.dual_value_lagrangian, dcopf.dual_value_prices):
        assert abs(fn(net, loads, lam, mh, ml) - d["gamma"]) < 1e-9
    can = dcopf.canonical(net, loads)
    assert abs(dcopf.dual_value_canonical_lp(can, lam, np.concatenate([mh, ml])) - d["gamma"]) < 1e-9


def test_three_bus_ptdf():
    net, _, d = hand("three_bus")
    e1 = np.array([0.0, 1.0, 0.0])
    e2 = np.array([0.0, 0.0, 1.0])
    assert np.allclose(net.flows(e1), d["ptdf_bus1"], atol=1e-14)
    assert np.allclose(net.flows(e2), d["ptdf_bus2"], atol=1e-14)
    phi = net.ptdf_gen()
    assert np.allclose(phi[:, 0], 0.0) and np.allclose(phi[:, 1], d["ptdf_bus2"])


def _node_branch_flows(net: dcopf.Net, y):
    """DC power flow from its two defining laws, solved as one least-squares system:
    KCL (inc^T f = y with the imbalance absorbed at the slack) and Ohm's law
    f_l = b_l (theta_from - theta_to), theta_slack = 0."""
    nb, nl = net.n_bus, net.n_line
    inc = np.zeros((nl, nb))
    inc[np.arange(nl), net.lf] = 1.0
    inc[np.arange(nl), net.lt] = -1.0
    yy = np.array(y, dtype=float)
    yy[net.slack] -= yy.sum()
    rows, rhs = [], []
    # unknowns: theta (nb), f (nl)
    for l in range(nl):
        r = np.zeros(nb + nl)
        r[net.lf[l]] = net.b[l]
        r[net.lt[l]] = -net.b[l]
        r[nb + l] = -1.0
        rows.append(r)
        rhs.append(0.0)
    for i in range(nb):
        r = np.zeros(nb + nl)
        r[nb:] = inc[:, i]
        rows.append(r)
        rhs.append(yy[i])
    r = np.zeros(nb + nl)
    r[net.slack] = 1.0
    rows.append(r)
    rhs.append(0.0)
    sol = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    return sol[nb:]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_flows_match_node_branch_and_adjoint(seed):
    s, _ = synth.tiny_network(seed, 9, 14, 3)
    net = onet(s)
    rng = np.random.default_rng(seed)
    y = rng.normal(size=net.n_bus)
    assert np.allclose(net.flows(y), _node_branch_flows(net, y), atol=1e-12)
    eta = rng.normal(size=net.n_line)
    # adjoint identity <eta, H_a y> = <H_a^T eta, y>
    assert abs(eta @ net.flows(y) - net.prices(eta) @ y) < 1e-12
    assert net.prices(eta)[net.slack] == 0.0


def test_merit_order_single_bus_lp():
    """No binding limits: gamma* is the merit-order cost and lambda* = -S c_marginal."""
    s, loads = synth.tiny_network(5, 8, 10, 5)
    d = s.as_dict()
    d["flow_max"] = np.full(s.n_line, 1e6)
    d["flow_min"] = -d["flow_max"]
    net = dcopf.Net.from_dict(d)
    order = np.argsort(net.c)
    rem, cost, marg = loads.sum(), 0.0, None
    for j in order:
        take = min(rem, net.pmax[j])
        cost += net.c[j] * net.S * take
        rem -= take
        if take > 0:
            marg = j
        if rem <= 0:
            break
    assert abs(exact.ipm(net, loads)["gamma"] - cost) < 1e-7 * cost
    assert abs(exact.vertex_enumeration(net, loads)[0] - cost) < 1e-9 * cost
    zero = np.zeros(net.n_line)
    lam = -net.c[marg] * net.S
    assert abs(dcopf.dual_value_prices(net, loads, lam, zero, zero) - cost) < 1e-9 * cost


def test_equal_incremental_cost_qp():
    """No binding limits, quadratic costs: bisection on lambda for
    sum_j clip((-lambda/S - b_j)/(2 a_j S), pmin, pmax) = D gives gamma*."""
    s, loads = synth.tiny_network(7, 10, 14, 6, quadratic=True)
    d = s.as_dict()
    d["flow_max"] = np.full(s.n_line, 1e6)
    d["flow_min"] = -d["flow_max"]
    net = dcopf.Net.from_dict(d)
    D = loads.sum()

    def disp(lam):
        return np.clip((-lam / net.S - net.c) / (2 * net.a * net.S), net.pmin, net.pmax)

    lo, hi = -1e6, 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if disp(mid).sum() > D:
            lo = mid
        else:
            hi = mid
    lam = 0.5 * (lo + hi)
    p = disp(lam)
    cost = float(np.sum(net.a * (net.S * p) ** 2 + net.c * net.S * p))
    assert abs(exact.ipm(net, loads)["gamma"] - cost) < 1e-8 * cost
    zero = np.zeros(net.n_line)
    assert abs(dcopf.dual_value_prices(net, loads, lam, zero, zero) - cost) < 1e-8 * cost


@pytest.mark.parametrize("seed", [11, 12, 13, 14, 15, 16])
def test_vertex_enumeration_matches_ipm(seed):
    s, loads = synth.tiny_network(seed, 5, 6, 4, tight=0.5)
    net = onet(s)
    gv, pv = exact.vertex_enumeration(net, loads)
    r = exact.ipm(net, loads)
    assert r["status"] == "optimal"
    assert abs(gv - r["gamma"]) < 1e-8 * abs(gv)
    try:
        from scipy.optimize import linprog
    except ImportError:
        return
    phi = net.ptdf_gen()
    fd = net.flows(loads)
    res = linprog(net.c * net.S, A_ub=np.vstack([phi, -phi]),
                  b_ub=np.concatenate([net.fmax + fd, -net.fmin - fd]),
                  A_eq=np.ones((1, net.n_gen)), b_eq=[loads.sum()],
                  bounds=list(zip(net.pmin, net.pmax)), method="highs")
    assert abs(res.fun - gv) < 1e-7 * abs(gv)


def _rand_point(rng, net, scale=200.0):
    return (-rng.uniform(1000, 5000), rng.exponential(scale, net.n_line) * (rng.random(net.n_line) < 0.3),
            rng.exponential(scale, net.n_line) * (rng.random(net.n_line) < 0.3))


@pytest.mark.parametrize("qp", [False, True])
def test_three_formulas_agree(qp):
    s, loads = synth.tiny_network(21, 30, 45, 8, quadratic=qp)
    net = onet(s)
    can = dcopf.canonical(net, loads)
    rng = np.random.default_rng(3)
    for _ in range(5):
        lam, mh, ml = _rand_point(rng, net)
        a = dcopf.dual_value_lagrangian(net, loads, lam, mh, ml)
        b = dcopf.dual_value_prices(net, loads, lam, mh, ml)
        assert abs(a - b) < 1e-12 * max(1.0, abs(a))
        mu = np.concatenate([mh, ml])
        if qp:
            _, _, _, p, _ = dcopf.dual_parts(net, loads, lam, mh, ml)
            x = (p - can["mid"]) / can["sigma"]
            s_star = -2.0 * np.sqrt(can["M"]) * x           # maximiser of eq. (16) over s
            c = dcopf.dual_value_canonical_qp(can, lam, mu, s_star)
            for _ in range(3):
                s_rand = s_star + rng.normal(scale=50.0, size=net.n_gen)
                assert dcopf.dual_value_canonical_qp(can, lam, mu, s_rand) <= c + 1e-9 * abs(c)
        else:
            c = dcopf.dual_value_canonical_lp(can, lam, mu)
        assert abs(a - c) < 1e-10 * max(1.0, abs(a))


@pytest.mark.parametrize("cfg_qp", [(0, False), (None, True)])
def test_weak_duality(cfg_qp):
    cfg, qp = cfg_qp
    if cfg is not None:
        s, loads = synth.network_for(cfg)
    else:
        s, loads = synth.tiny_network(31, 40, 60, 10, quadratic=qp)
    net = onet(s)
    r = exact.ipm(net, loads)
    assert r["status"] == "optimal"
    # proportional base dispatch is feasible by construction of the limits
    p_base = net.pmax * loads.sum() / net.pmax.sum()
    ub_feasible = net.cost(p_base)
    rng = np.random.default_rng(5)
    for _ in range(20):
        lam, mh, ml = _rand_point(rng, net)
        g = dcopf.dual_value_prices(net, loads, lam, mh, ml)
        assert g <= r["ub"] + 1e-9 * abs(r["ub"])
        assert g <= ub_feasible
    assert r["lb"] <= ub_feasible


@pytest.mark.parametrize("qp", [False, True])
def test_concavity_supergradient(qp):
    s, loads = synth.tiny_network(41, 25, 36, 7, quadratic=qp)
    net = onet(s)
    rng = np.random.default_rng(8)
    for _ in range(10):
        lam, mh, ml = _rand_point(rng, net)
        val, gl, ghi, glo, _ = dcopf.evaluate(net, loads, lam, mh, ml)
        dl = rng.normal(scale=300.0)
        dh = rng.normal(scale=100.0, size=net.n_line)
        dlo = rng.normal(scale=100.0, size=net.n_line)
        v2 = dcopf.dual_value_lagrangian(net, loads, lam + dl, mh + dh, ml + dlo)
        assert v2 <= val + gl * dl + ghi @ dh + glo @ dlo + 1e-9 * abs(val)


def test_finite_differences_qp():
    s, loads = synth.tiny_network(51, 20, 30, 6, quadratic=True)
    net = onet(s)
    rng = np.random.default_rng(9)
    lam, mh, ml = _rand_point(rng, net, scale=20.0)
    val, gl, ghi, glo, _ = dcopf.evaluate(net, loads, lam, mh, ml)
    h = 1e-3
    fl = (dcopf.dual_value_lagrangian(net, loads, lam + h, mh, ml)
          - dcopf.dual_value_lagrangian(net, loads, lam - h, mh, ml)) / (2 * h)
    assert abs(fl - gl) < 1e-5 * max(1.0, abs(gl))
    for i in rng.choice(net.n_line, 5, replace=False):
        e = np.zeros(net.n_line)
        e[i] = h
        fh = (dcopf.dual_value_lagrangian(net, loads, lam, mh + e, ml)
              - dcopf.dual_value_lagrangian(net, loads, lam, mh - e, ml)) / (2 * h)
        assert abs(fh - ghi[i]) < 1e-5 * max(1.0, abs(ghi[i]))


def test_slack_invariance_of_gamma():
    s, loads = synth.tiny_network(61, 12, 18, 4, tight=0.5)
    d = s.as_dict()
    g0 = exact.ipm(dcopf.Net.from_dict(d), loads)["gamma"]
    d["slack_bus"] = 7
    g7 = exact.ipm(dcopf.Net.from_dict(d), loads)["gamma"]
    assert abs(g0 - g7) < 1e-9 * abs(g0)


def test_ascent_rules_first_steps():
    """Iterates of each rule from the cold start (Algorithm 1, Require), by hand:
    GDM (heavy ball): v1 = alpha g0, theta1 = v1; v2 = rho v1 + alpha g1, theta2 = theta1 + v2.
    Adam: first step alpha * m1_hat / sqrt(v1_hat) = alpha * sign(g0).
    AdaGrad: first step alpha * g0 / |g0| = alpha * sign(g0).
    mu is projected to max(mu, 0) after every step."""
    net, loads, _ = hand("two_bus")
    z = np.zeros(1)
    _, gl0, ghi0, glo0, _ = dcopf.evaluate(net, loads, 0.0, z, z)
    a, rho = 2.0, 0.5
    # GDM, two steps
    r = dcopf.solve(net, loads, rule="gdm", alpha=a, rho=rho, max_iters=3, record=True)
    l1, h1, o1 = a * gl0, np.maximum(a * ghi0, 0), np.maximum(a * glo0, 0)
    assert abs(r["points"][1][0] - l1) < 1e-12 and np.allclose(r["points"][1][1], h1)
    _, gl1, ghi1, glo1, _ = dcopf.evaluate(net, loads, l1, h1, o1)
    l2 = l1 + rho * a * gl0 + a * gl1
    h2 = np.maximum(h1 + rho * a * ghi0 + a * ghi1, 0)
    assert abs(r["points"][2][0] - l2) < 1e-9 and np.allclose(r["points"][2][1], h2)
    # as printed: theta1 = 2 alpha g0
    r = dcopf.solve(net, loads, rule="gdm", alpha=a, rho=rho, max_iters=2, record=True,
                    as_printed=True)
    assert abs(r["points"][1][0] - 2 * a * gl0) < 1e-12
    for rule in ("adam", "adagrad"):
        r = dcopf.solve(net, loads, rule=rule, alpha=a, eps=0.0, max_iters=2, record=True)
        assert abs(r["points"][1][0] - a * np.sign(gl0)) < 1e-12
        assert np.allclose(r["points"][1][1], np.maximum(a * np.sign(ghi0), 0))
    # Adam second step with bias correction, lambda coordinate
    b1, b2 = 0.9, 0.99
    r = dcopf.solve(net, loads, rule="adam", alpha=a, beta1=b1, beta2=b2, eps=0.0, max_iters=3,
                    record=True)
    lam1, mh1, ml1 = r["points"][1]
    _, gl1, _, _, _ = dcopf.evaluate(net, loads, lam1, mh1, ml1)
    m = (1 - b1) * (b1 * gl0 + gl1)
    v = (1 - b2) * (b2 * gl0 ** 2 + gl1 ** 2)
    step = a * (m / (1 - b1 ** 2)) / np.sqrt(v / (1 - b2 ** 2))
    assert abs(r["points"][2][0] - (lam1 + step)) < 1e-9


def test_adam_converges_on_hand_and_c0():
    for net, loads in (hand("three_bus")[:2], (onet(synth.network_for(0)[0]), synth.network_for(0)[1])):
        g = exact.ipm(net, loads)["gamma"]
        r = dcopf.solve(net, loads, rule="adam", alpha=1000.0 if net.S > 1 else 1.0,
                        beta1=0.9, beta2=0.999, decay=0.99, max_iters=5000, target=g, gap=1e-3)
        assert r["stop"] == "target"
        assert g * (1 - 1e-3) - 1e-9 <= r["best"] <= g + 1e-9 * abs(g)


def test_ascent_rules_decay_and_alpha_lambda():
    """Decayed steps with a separate lambda step size, written out by hand.

    Step-size decay (Section 4.1 remarks) is read as a multiplicative schedule: the k-th
    step (k = 1, 2, ...) uses alpha * decay^(k-1) for mu and alpha_lambda * decay^(k-1)
    for lambda.  Three GDM steps (heavy ball, the velocity keeps the undecayed earlier
    contributions), two Adam steps and two AdaGrad steps (the second divides by the
    root of the summed squares of both gradients)."""
    net, loads, _ = hand("three_bus")
    z = np.zeros(net.n_line)
    a, al, rho, d = 3.0, 0.5, 0.6, 0.8

    def grad(lam, mh, ml):
        _, gl, ghi, glo, _ = dcopf.evaluate(net, loads, lam, mh, ml)
        return gl, ghi, glo

    # GDM: v_k = rho v_{k-1} + step_k g_{k-1}, theta_k = theta_{k-1} + v_k, mu projected
    r = dcopf.solve(net, loads, rule="gdm", alpha=a, alpha_lambda=al, rho=rho, decay=d,
                    max_iters=4, record=True)
    lam, mh, ml = 0.0, z.copy(), z.copy()
    vl, vh, vo = 0.0, z.copy(), z.copy()
    for k in (1, 2, 3):
        gl, ghi, glo = grad(lam, mh, ml)
        vl = rho * vl + al * d ** (k - 1) * gl
        vh = rho * vh + a * d ** (k - 1) * ghi
        vo = rho * vo + a * d ** (k - 1) * glo
        lam, mh, ml = lam + vl, np.maximum(mh + vh, 0), np.maximum(ml + vo, 0)
        pl, ph, po = r["points"][k]
        assert abs(pl - lam) < 1e-12 * max(1.0, abs(lam))
        assert np.allclose(ph, mh, rtol=1e-12, atol=1e-12)
        assert np.allclose(po, ml, rtol=1e-12, atol=1e-12)
    assert abs(r["points"][1][0] - al * grad(0.0, z, z)[0]) < 1e-12   # undecayed first step

    # Adam, eps = 0: first step alpha_lambda sign(g0); second step decayed
    b1, b2 = 0.7, 0.9
    r = dcopf.solve(net, loads, rule="adam", alpha=a, alpha_lambda=al, beta1=b1, beta2=b2,
                    eps=0.0, decay=d, max_iters=3, record=True)
    gl0, ghi0, _ = grad(0.0, z, z)
    lam1, mh1, ml1 = r["points"][1]
    assert abs(lam1 - al * np.sign(gl0)) < 1e-12
    assert np.allclose(mh1, np.maximum(a * np.sign(ghi0), 0))
    gl1, ghi1, _ = grad(lam1, mh1, ml1)
    m = (1 - b1) * (b1 * gl0 + gl1) / (1 - b1 ** 2)
    v = (1 - b2) * (b2 * gl0 ** 2 + gl1 ** 2) / (1 - b2 ** 2)
    assert abs(r["points"][2][0] - (lam1 + al * d * m / np.sqrt(v))) < 1e-9
    mv = (1 - b1) * (b1 * ghi0 + ghi1) / (1 - b1 ** 2)
    vv = (1 - b2) * (b2 * ghi0 ** 2 + ghi1 ** 2) / (1 - b2 ** 2)
    nz = vv > 0
    want = mh1.copy()
    want[nz] = np.maximum(mh1[nz] + a * d * mv[nz] / np.sqrt(vv[nz]), 0)
    assert np.allclose(r["points"][2][1], want, rtol=1e-12, atol=1e-9)

    # AdaGrad, eps = 0: theta_2 = theta_1 + step_2 g1 / sqrt(g0^2 + g1^2)
    r = dcopf.solve(net, loads, rule="adagrad", alpha=a, alpha_lambda=al, eps=0.0, decay=d,
                    max_iters=3, record=True)
    lam1, mh1, ml1 = r["points"][1]
    assert abs(lam1 - al * np.sign(gl0)) < 1e-12
    gl1, ghi1, _ = grad(lam1, mh1, ml1)
    assert abs(r["points"][2][0] - (lam1 + al * d * gl1 / np.sqrt(gl0 ** 2 + gl1 ** 2))) < 1e-12
    den = np.sqrt(ghi0 ** 2 + ghi1 ** 2)
    want = mh1.copy()
    want[den > 0] = np.maximum(mh1[den > 0] + a * d * ghi1[den > 0] / den[den > 0], 0)
    assert np.allclose(r["points"][2][1], want, rtol=1e-12, atol=1e-12)


def test_qp_dual_with_s_variable():
    """Eq. (16) with s as an ascent variable (Remark 2): at s = -2 sqrt(M) x* it equals the
    closed-form dual (minimax), any other s gives less; its s-gradient -sqrt(M) x* - s/2
    matches central finite differences where no reduced cost ties; the first Adam step
    from the cold start moves every coordinate by alpha sign(gradient), written out by
    hand; and the s-ascent reaches the 0.1 % gap on a small QP, its in-loop value g_q
    staying below the certified closed-form value."""
    s_, loads = synth.tiny_network(23, 16, 24, 6, quadratic=True)
    net = onet(s_)
    can = dcopf.canonical(net, loads)
    rng = np.random.default_rng(12)
    lam, mh, ml = _rand_point(rng, net, scale=20.0)
    sv = rng.normal(scale=30.0, size=net.n_gen)
    val, gl, gh, go, gs, p = dcopf.evaluate_qp_s(net, can, loads, lam, mh, ml, sv)
    x = (p - can["mid"]) / can["sigma"]
    sq = np.sqrt(can["M"])
    assert np.all(np.isin(np.round(x, 12), [-1.0, 1.0]))
    closed = dcopf.dual_value_prices(net, loads, lam, mh, ml)
    assert val <= closed + 1e-9 * abs(closed)
    h = 1e-4
    for j in range(net.n_gen):
        e = np.zeros(net.n_gen)
        e[j] = h
        fd = (dcopf.evaluate_qp_s(net, can, loads, lam, mh, ml, sv + e)[0]
              - dcopf.evaluate_qp_s(net, can, loads, lam, mh, ml, sv - e)[0]) / (2 * h)
        assert abs(fd - gs[j]) < 1e-5 * max(1.0, abs(gs[j]))
    assert abs(gs[0] - (-sq[0] * x[0] - 0.5 * sv[0])) < 1e-12 * max(1.0, abs(gs[0]))
    # first Adam step, eps = 0: theta_1 = alpha * sign(g_0)
    a = 2.0
    r = dcopf.solve_qp_s(net, loads, rule="adam", alpha=a, eps=0.0, max_iters=2, record=True)
    z = np.zeros(net.n_line)
    _, gl0, gh0, _, gs0, _ = dcopf.evaluate_qp_s(net, can, loads, 0.0, z, z, np.zeros(net.n_gen))
    p1 = r["points"][1]
    assert abs(p1["lam"][0] - a * np.sign(gl0)) < 1e-12
    assert np.allclose(p1["s"], a * np.sign(gs0)) and np.allclose(p1["mh"], np.maximum(a * np.sign(gh0), 0))
    # convergence to the gap (certified through the closed form at (lambda, mu))
    gam = exact.ipm(net, loads)["gamma"]
    r = dcopf.solve_qp_s(net, loads, rule="adam", alpha=1000.0, beta1=0.9, beta2=0.999, decay=0.998,
                         max_iters=5000, target=gam, gap=1e-3)
    assert r["iters"] < 5000
    assert gam * (1 - 1e-3) - 1e-9 * abs(gam) <= r["best_closed"] <= gam + 1e-9 * abs(gam)
    assert r["best"] <= r["best_closed"] + 1e-9 * abs(gam)


@pytest.mark.parametrize("seed", [0, 1])
def test_outage_network_matches_lodf_identity(seed):
    """The post-outage reference of the GPU outage tests (the network rebuilt without
    line k) against the textbook line-outage distribution factor: for an injection y,
    f'_l = f_l + LODF_lk f_k with LODF_lk = PTDF_l,(a->c) / (1 - PTDF_k,(a->c)), where
    PTDF_.,(a->c) are the full network's flows of a unit transfer from line k's from-bus
    a to its to-bus c.  Also: the two-bus closed form PTDF = 1 of a lone line."""
    from gpu_common import drop_line
    net, base = synth.network_for(0)
    on = onet(net)
    rng = np.random.default_rng(seed)
    # non-bridge lines: removing one leaves the network connected (finite LODF)
    for k in rng.permutation(net.n_line)[:6]:
        a, c = int(net.line_from[k]), int(net.line_to[k])
        t = np.zeros(net.n_bus)
        t[a], t[c] = 1.0, -1.0
        ptdf_t = on.flows(t)
        if abs(1.0 - ptdf_t[k]) < 1e-9:
            continue   # a bridge
        y = base * rng.uniform(0.8, 1.2, net.n_bus)
        y[on.slack] -= y.sum()                       # balanced injection
        f = on.flows(y)
        lodf = ptdf_t / (1.0 - ptdf_t[k])
        expect = np.delete(f + lodf * f[k], k)
        got = drop_line(net, int(k)).flows(y)
        assert np.allclose(got, expect, rtol=1e-10, atol=1e-10 * np.max(np.abs(f)))
    two = dcopf.Net(2, [0], [1], [5.0], [1.0], None, [0], [0.0], [1.0], [1.0], None, base_mva=1.0)
    assert abs(two.flows(np.array([1.0, -1.0]))[0] - 1.0) <= 1e-15
