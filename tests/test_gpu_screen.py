"""Constraint screening (the rows C_r, d_r of Algorithm 1 read as the flow rows that can
bind) on the batched tensor-core path.

A screened line must be one whose flow stays inside its limits for every dispatch of the
generator box that meets the balance, at every instance's loads.  The oracle side checks
that with its own fractional knapsack per line and instance: generators sorted by their
flow coefficient, filled greedily from the box's lower end to the demand (the exact
maximum of a linear function over the box and one equality).  Screened solves then reach
the certified gap with valid bounds; since a screened line's flow gradient is negative
at every point, its multipliers stay zero from a cold start and the iterations follow
the unscreened ones (up to the rounding of sums over fewer rows).
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2406_13191_gb300 import DcopfDual, synth

from gpu_common import gamma, onet

pytestmark = pytest.mark.gpu

ADAM_QP = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000)
ADAM_LP = dict(rule="adam", alpha=1000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=6000)


def knapsack_flow_range(phi_row, pmin, pmax, D, fd):
    """Exact max and min of phi_row . p - fd over pmin <= p <= pmax, sum p = D: start at
    pmin and raise generators in order of decreasing (max) or increasing (min) coefficient
    until the demand is met."""
    out = []
    for order in (np.argsort(-phi_row), np.argsort(phi_row)):
        p = pmin.copy()
        rem = D - pmin.sum()
        for j in order:
            take = min(pmax[j] - pmin[j], rem)
            p[j] += take
            rem -= take
            if rem <= 0:
                break
        out.append(float(phi_row @ p - fd))
    return out[0], out[1]


@pytest.mark.parametrize("quadratic", [False, True])
def test_screen_drops_only_lines_that_cannot_bind(quadratic):
    w = synth.scenario_workload(81, 80, 130, 14, quadratic, batch=40, n_out=0)
    on = onet(w.net)
    g = DcopfDual(w.net)
    gams = [gamma(on, w.loads[b]) for b in range(w.batch)]
    kw = ADAM_QP if quadratic else ADAM_LP
    r0 = g.solve(w.loads, path="batched", precision="bf16x3", target=gams, **kw)
    st0, it0 = r0.status.cpu().numpy(), r0.iters.cpu().numpy()
    res = g.solve(w.loads, path="batched", precision="bf16x3", target=gams, screen=True, **kw)
    torch.cuda.synchronize()
    kept = g.screened_lines()
    assert kept.any() and kept.sum() % 8 == 0
    phi = on.ptdf_gen()
    exact_free = np.ones(on.n_line, dtype=bool)   # lines that stay strictly inside for every instance
    for b in range(w.batch):
        fd = on.flows(w.loads[b])
        D = w.loads[b].sum()
        for l in range(on.n_line):
            hi, lo = knapsack_flow_range(phi[l], on.pmin, on.pmax, D, fd[l])
            if not (hi < on.fmax[l] and lo > on.fmin[l]):
                exact_free[l] = False
    assert not np.any(~kept & ~exact_free), np.flatnonzero(~kept & ~exact_free)
    print(f"{'QP' if quadratic else 'LP'}: {on.n_line} lines, {exact_free.sum()} cannot bind, "
          f"{(~kept).sum()} screened, {kept.sum()} kept")
    # the screened solve reaches the gap where the unscreened one does, in about as many
    # iterations, and every bound is valid
    st1, it1 = res.status.cpu().numpy(), res.iters.cpu().numpy()
    both = (st0 == 0) & (st1 == 0)
    assert (st1 == 0).sum() >= (st0 == 0).sum() - max(1, w.batch // 20), (st0, st1)
    assert abs(it1[both].mean() - it0[both].mean()) <= 0.1 * it0[both].mean()
    for b in range(w.batch):
        bnd = res.bound[b].item()
        assert bnd <= gams[b] + 1e-9 * abs(gams[b])
        if st1[b] == 0:
            assert gams[b] * (1 - 1e-3) - 1e-9 * abs(gams[b]) <= bnd
        assert np.all(res.mu_hi[b].cpu().numpy()[~kept] == 0.0)
    print(f"  reached: {(st0 == 0).sum()} unscreened, {(st1 == 0).sum()} screened of {w.batch}; "
          f"iterations {it0[both].mean():.1f} / {it1[both].mean():.1f}")


def test_screened_10000bus_batch_reaches_stored_optima():
    """64 instances of the 10000-bus batch with and without screening: every bound valid
    and within the gap, and the same iterations up to rounding."""
    gam = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c3_gamma.json")))["gamma"][:64]
    w = synth.workload(3, batch=64)
    g = DcopfDual(w.net)
    T = np.array(gam)
    r0 = g.solve(w.loads, path="batched", precision="bf16x3", target=T, **ADAM_QP)
    it0 = r0.iters.cpu().numpy()
    r1 = g.solve(w.loads, path="batched", precision="bf16x3", target=T, screen=True, **ADAM_QP)
    torch.cuda.synchronize()
    kept = g.screened_lines()
    b1 = r1.bound.cpu().numpy()
    assert (r1.status.cpu().numpy() == 0).all()
    assert np.all(b1 <= T + 1e-9 * np.abs(T)) and np.all(b1 >= T * (1 - 1e-3) - 1e-9 * np.abs(T))
    it1 = r1.iters.cpu().numpy()
    assert abs(it1.mean() - it0.mean()) <= 0.05 * it0.mean()
    print(f"10000-bus: {kept.sum()} of {w.net.n_line} lines kept; iterations {it0.mean():.1f} "
          f"unscreened, {it1.mean():.1f} screened")


def test_speculative_screen_rescreens_a_batch_that_needs_more_lines(monkeypatch):
    """A handle goes ahead with its last kept set when a new batch comes; the solve then
    learns on the device whether the batch needs a line outside it and, if so, runs
    again with the batch's own screen.  A batch of 16 copies of 0.85 x the mean load, then
    16 scenarios of the workload: the second must keep lines the first screened out, and
    its solve on the reused handle equals the solve of the same batch on a fresh handle."""
    w = synth.scenario_workload(81, 80, 130, 14, True, batch=40, n_out=0)
    on = onet(w.net)
    base = w.loads.mean(axis=0)
    narrow = np.repeat(0.85 * base[None], 16, 0)
    wide = w.loads[:16]
    gam_w = [gamma(on, wide[b]) for b in range(16)]
    gam_n = [gamma(on, narrow[b]) for b in range(16)]
    kw = dict(path="batched", precision="bf16x3", screen=True, **ADAM_QP)
    monkeypatch.setenv("DCOPF_TENSOR_SHAPE", "0,2,0,1")   # the same product shapes on both handles
    g = DcopfDual(w.net)
    g.solve(narrow, target=gam_n, **kw)
    kept_n = g.screened_lines()
    r = g.solve(wide, target=gam_w, **kw)
    torch.cuda.synchronize()
    kept_w = g.screened_lines()
    f = DcopfDual(w.net)
    monkeypatch.delenv("DCOPF_TENSOR_SHAPE")
    rf = f.solve(wide, target=gam_w, **kw)
    torch.cuda.synchronize()
    kept_f = f.screened_lines()
    print(f"kept: {kept_n.sum()} narrow, {kept_f.sum()} wide (fresh), {kept_w.sum()} wide (reused)")
    assert np.any(kept_f & ~kept_n), "the wide batch should need a line the narrow one screens out"
    np.testing.assert_array_equal(kept_w, kept_f)
    for a, b in ((r.bound, rf.bound), (r.iters, rf.iters), (r.status, rf.status), (r.lam, rf.lam)):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert np.all(r.bound.cpu().numpy() <= np.array(gam_w) + 1e-9 * np.abs(gam_w))
