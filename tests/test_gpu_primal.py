"""GPU parity of the primal recovery (dcopf_dual_primal_bound, csrc/k_primal.cu)
against the oracle's (oracle/primal.py), on seeded networks of assorted sizes, LP and
QP, with and without line outages.

Outage instances are compared with the oracle on the network rebuilt without the
line. Tolerances: the status exactly; the upper bound to 1e-9 relative (both FP64;
the bisections bracket the same shift with differently rounded prices); the
dispatch to 1e-7 of the largest |p| (a unit whose price threshold lies within
rounding of the bracketed shift may be interpolated differently); the recomputed
flow violation below 1e-9 p.u.
"""
import numpy as np
import pytest

from oracle import dcopf, exact, primal
from paper_2406_13191_gb300 import DcopfDual, synth

from gpu_common import drop_line, onet, rand_point

pytestmark = pytest.mark.gpu

# (seed, buses, lines, generators, quadratic, instances, outages)
CASES = [(201, 23, 31, 4, False, 6, 2), (202, 57, 80, 13, True, 6, 3),
         (203, 140, 190, 31, True, 8, 3), (204, 96, 150, 9, False, 6, 2),
         (205, 210, 300, 70, True, 8, 4)]


def _points(rng, nl, B, outage):
    """Dual points of three kinds: mu = 0 (uniform prices), small and large random
    multipliers; the outaged line carries none."""
    lam, mh, ml = [], [], []
    for b in range(B):
        kind = b % 3
        if kind == 0:
            p = (-rng.uniform(1000, 5000), np.zeros(nl), np.zeros(nl))
        else:
            p = rand_point(rng, nl, scale=30.0 if kind == 1 else 300.0)
        if outage[b] >= 0:
            p[1][outage[b]] = p[2][outage[b]] = 0.0
        lam.append(p[0])
        mh.append(p[1])
        ml.append(p[2])
    return np.array(lam), np.stack(mh), np.stack(ml)


def _check(b, ub, st, disp, viol, r):
    assert int(st) == r["status"], (b, int(st), r["status"])
    if r["status"] != 0:
        assert ub == np.inf and np.all(np.isnan(disp))
        return
    assert abs(ub - r["ub"]) <= 1e-9 * abs(r["ub"]), (b, ub, r["ub"])
    assert np.max(np.abs(disp - r["p"])) <= 1e-7 * max(1.0, np.max(np.abs(r["p"])))
    assert viol <= 1e-9


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[1]}" for c in CASES])
def test_primal_bound_matches_oracle(case):
    seed, nb, nl, ng, qp, B, n_out = case
    w = synth.scenario_workload(seed, nb, nl, ng, qp, batch=B, n_out=n_out)
    g = DcopfDual(w.net)
    lam, mh, ml = _points(np.random.default_rng(seed), nl, B, w.outage)
    ub, st, disp, viol = (t.cpu().numpy() for t in g.primal_bound(w.loads, lam, mh, ml, outage=w.outage))
    on = onet(w.net)
    seen = set()
    for b in range(B):
        k = int(w.outage[b])
        o = on if k < 0 else drop_line(w.net, k)
        keep = np.arange(nl) != k
        r = primal.recover(o, w.loads[b], lam[b], mh[b][keep], ml[b][keep])
        _check(b, ub[b], st[b], disp[b], viol[b], r)
        seen.add(r["status"])
    assert 0 in seen   # the comparison covered recovered bounds


def test_caller_reference_and_statuses():
    """A caller's reference (the oracle's optimum of each instance) is used as given;
    an unbalanced one and a demand beyond the box are reported, not bounded."""
    w = synth.scenario_workload(206, 60, 90, 12, True, batch=4, n_out=0)
    g = DcopfDual(w.net)
    on = onet(w.net)
    rng = np.random.default_rng(5)
    lam, mh, ml = _points(rng, w.net.n_line, 4, w.outage)
    opt = [exact.ipm(on, w.loads[b]) for b in range(4)]
    p_ref = np.stack([o["p"] for o in opt])
    p_ref[3] *= 1.01                               # unbalanced: no bound
    ub, st, disp, viol = (t.cpu().numpy() for t in g.primal_bound(w.loads, lam, mh, ml, p_ref=p_ref))
    for b in range(4):
        r = primal.recover(on, w.loads[b], lam[b], mh[b], ml[b], p_ref=p_ref[b])
        _check(b, ub[b], st[b], disp[b], viol[b], r)
        if b < 3:
            assert st[b] == 0 and ub[b] >= opt[b]["gamma"] * (1 - 1e-9)
    assert st[3] == 2
    big = w.loads * 50.0                           # beyond sum pmax
    ub, st, _, _ = g.primal_bound(big[:1], lam[:1], mh[:1], ml[:1])
    assert int(st[0]) == 1 and ub[0].item() == np.inf


def test_gap_without_an_oracle_after_a_solve():
    """After a solve to the certified 0.1 % gap on the 120-bus QP stand-in, the
    recovered dispatch is feasible and its cost brackets gamma* with the bound."""
    w = synth.scenario_workload(207, 120, 170, 25, True, batch=6, n_out=0)
    g = DcopfDual(w.net)
    on = onet(w.net)
    gam = np.array([exact.ipm(on, w.loads[b])["gamma"] for b in range(6)])
    r = g.solve(w.loads, target=gam, rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999,
                decay=0.997, max_iters=4000, path="batched", precision="bf16x3")
    lb = r.bound.cpu().numpy()
    ub, st, disp, viol = (t.cpu().numpy() for t in g.primal_bound(w.loads, r.lam, r.mu_hi, r.mu_lo))
    assert np.all(st == 0) and np.all(viol <= 1e-9)
    assert np.all(lb <= gam * (1 + 1e-12)) and np.all(ub >= gam * (1 - 1e-12))
    assert np.all((ub - lb) / ub < 0.5)


def test_recovery_from_a_candidate_matches_oracle():
    """p_cand replaces the minimiser: the oracle's k^2-weighted mean of the minimisers
    of its own solve, balanced and repaired on both sides; FP64 parity as above."""
    w = synth.scenario_workload(208, 90, 130, 18, True, batch=3, n_out=0)
    g = DcopfDual(w.net)
    on = onet(w.net)
    cands, recs = [], []
    for b in range(3):
        r = dcopf_solve(on, w.loads[b])
        cands.append(r["mean_dispatch"])
        recs.append(primal.recover(on, w.loads[b], None, None, None, p_cand=r["mean_dispatch"]))
    ub, st, disp, viol = (t.cpu().numpy() for t in g.primal_bound(w.loads, p_cand=np.stack(cands)))
    for b in range(3):
        _check(b, ub[b], st[b], disp[b], viol[b], recs[b])
    assert np.all(st == 0)


def dcopf_solve(on, loads):
    return dcopf.solve(on, loads, rule="adam", alpha=1000.0, beta1=0.95, beta2=0.999, max_iters=60)


@pytest.mark.parametrize("path", ["plain", "sparse"])
def test_mean_dispatch_of_the_fp64_paths_follows_the_oracle(path):
    """The plain and sparse FP64 paths evaluate the oracle's points (test_gpu_solve), so
    their mean of the minimisers (FP32 sums of k^2 x) agrees with the oracle's to FP32
    rounding."""
    w = synth.scenario_workload(209, 70, 100, 15, True, batch=1, n_out=0)
    g = DcopfDual(w.net)
    on = onet(w.net)
    kw = dict(rule="gdm", alpha=10.0, alpha_lambda=0.1, rho=0.995, max_iters=40)
    res = g.solve(w.loads, path=path, precision="fp64", mean_dispatch=True, **kw)
    ref = dcopf.solve(on, w.loads[0], **kw)
    assert res.iters[0].item() == 40
    md = res.mean_dispatch[0].cpu().numpy()
    assert np.max(np.abs(md - ref["mean_dispatch"])) <= 1e-5 * max(1.0, np.max(np.abs(md)))


@pytest.mark.parametrize("path", ["fused", "batched"])
def test_mean_dispatch_gives_valid_bounds(path):
    """The fused and batched paths return the mean of their minimisers (in the box); the
    bound recovered from it is feasible and above gamma*."""
    w = synth.scenario_workload(210, 120, 170, 25, True, batch=1 if path == "fused" else 5, n_out=0)
    g = DcopfDual(w.net)
    on = onet(w.net)
    B = w.loads.shape[0]
    gam = np.array([exact.ipm(on, w.loads[b])["gamma"] for b in range(B)])
    r = g.solve(w.loads, target=gam, rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999,
                decay=0.997, max_iters=4000, path=path,
                precision="fp32" if path == "fused" else "bf16x3", mean_dispatch=True)
    md = r.mean_dispatch.cpu().numpy()
    pmin, pmax = np.asarray(w.net.pmin), np.asarray(w.net.pmax)
    assert np.all(md >= pmin - 1e-6) and np.all(md <= pmax + 1e-6)
    ub, st, disp, viol = (t.cpu().numpy() for t in g.primal_bound(w.loads, p_cand=r.mean_dispatch))
    assert np.all(st == 0) and np.all(viol <= 1e-9)
    assert np.all(ub >= gam * (1 - 1e-12))
