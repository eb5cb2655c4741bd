"""Ascent trajectories of every solve path against the oracle, with step decay.

The oracle's schedule (tests/test_oracle_pins.py, test_ascent_rules_decay_and_alpha_lambda)
is the k-th step taking alpha decay^(k-1) for mu and alpha_lambda decay^(k-1) for
lambda (Section 4.1's step decay read as a multiplicative schedule; Algorithm 1 for
GDM, Adam and AdaGrad as in Section 3.3).  Each path runs a fixed number of
iterations without a target and returns its best iterate; the oracle runs the same
iterations in FP64 from the same cold start.

Bar, per instance:
  - FP64 paths (plain, sparse): lambda and the best value to 1e-8 relative.
  - FP32 and BF16x3 operator products: lambda to 1e-5 relative and the best value
    to 1e-4 relative.  The operator products carry relative errors of about 1e-7
    (FP32) and 4e-6 (three BF16 split products drop the lo*lo term, 2^-18 of each
    product).  The fused kernel also carries the ascent direction and moments of
    lambda in FP32: each step is then off by a few 2^-24 of its size, at most
    alpha_lambda (1 - beta1) / sqrt(1 - beta2) ~ 1.6 alpha_lambda for Adam, so 30
    steps of the settings below (alpha_lambda 400, |lambda| ~ 1e3) move lambda by up
    to about 4e-6 of its size.  A wrong schedule moves it far more: one decay factor
    too many or too few on every step shifts lambda by about 1e-2 here, and alpha in
    place of alpha_lambda by more.
The returned point is the best iterate.  Where several iterates' oracle values lie
within the value bar of the best, any of them is a correct answer, so lambda is
compared with the nearest of those.
"""
import numpy as np
import pytest
import torch

from oracle import dcopf
from paper_2406_13191_gb300 import DcopfDual, synth

from gpu_common import drop_line, onet

pytestmark = pytest.mark.gpu

ITERS = 30
RULES = {
    "gdm": dict(rule="gdm", alpha=10.0, alpha_lambda=0.1, rho=0.9, decay=0.99),
    "adam": dict(rule="adam", alpha=1000.0, alpha_lambda=400.0, beta1=0.95, beta2=0.999,
                 decay=0.99),
    "adagrad": dict(rule="adagrad", alpha=1000.0, alpha_lambda=300.0, decay=0.99),
}


def _compare(res, b, on, loads, kw, rtol_lam, rtol_val, keep=None):
    ref = dcopf.solve(on, loads, max_iters=ITERS, record=True, **kw)
    assert res.iters[b].item() == ITERS and res.status[b].item() == 1
    hist = ref["history"]
    best = ref["best"]
    bnd = res.bound[b].item()
    err_val = abs(bnd - best) / abs(best)
    assert err_val <= rtol_val, (b, bnd, best, err_val)
    near = np.flatnonzero(hist >= best - 2 * rtol_val * abs(best))
    lam = res.lam[b].item()
    err_lam = min(abs(lam - ref["points"][i][0]) / abs(ref["points"][i][0]) for i in near)
    assert err_lam <= rtol_lam, (b, lam, [ref["points"][i][0] for i in near], err_lam)
    if len(near) == 1:
        mh = res.mu_hi[b].cpu().numpy()
        if keep is not None:
            mh = mh[keep]
        scale = max(1.0, float(np.max(np.abs(ref["mu_hi"]))))
        assert np.max(np.abs(np.maximum(mh, 0) - ref["mu_hi"])) <= 10 * rtol_lam * scale
    return err_lam, err_val


@pytest.fixture(scope="module")
def c1():
    net, base = synth.network_for(1)
    return net, base, onet(net), DcopfDual(net)


@pytest.mark.parametrize("rule", ["gdm", "adam", "adagrad"])
@pytest.mark.parametrize("path", ["plain", "sparse"])
def test_fp64_paths_follow_oracle_with_decay(c1, path, rule):
    net, base, on, g = c1
    kw = RULES[rule]
    res = g.solve(base[None], path=path, precision="fp64", max_iters=ITERS, **kw)
    torch.cuda.synchronize()
    el, ev = _compare(res, 0, on, base, kw, 1e-8, 1e-8)
    print(f"{path} {rule}: lambda rel err {el:.2e}, value {ev:.2e}")


@pytest.mark.parametrize("rule", ["gdm", "adam", "adagrad"])
def test_fused_follows_oracle_with_decay(c1, rule):
    net, base, on, g = c1
    kw = RULES[rule]
    res = g.solve(base[None], path="fused", precision="fp32", max_iters=ITERS, **kw)
    torch.cuda.synchronize()
    el, ev = _compare(res, 0, on, base, kw, 1e-5, 1e-4)
    print(f"fused {rule}: lambda rel err {el:.2e}, value {ev:.2e}")


@pytest.fixture(scope="module")
def scen130():
    """130 load scenarios of a 60-bus QP network, 40 with a line outage: the batch
    crosses the 128-instance row tile of the tensor path, with a ragged last tile."""
    w = synth.scenario_workload(79, 60, 90, 12, True, batch=130, n_out=40)
    on = onet(w.net)
    nets = [on if w.outage[b] < 0 else drop_line(w.net, int(w.outage[b])) for b in range(w.batch)]
    return w, nets, DcopfDual(w.net)


@pytest.mark.parametrize("rule", ["gdm", "adam"])
@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_batched_follows_oracle_with_decay(scen130, precision, rule):
    w, nets, g = scen130
    kw = RULES[rule]
    res = g.solve(w.loads, outage=w.outage, path="batched", precision=precision,
                  max_iters=ITERS, **kw)
    torch.cuda.synchronize()
    worst_l = worst_v = 0.0
    for b in range(w.batch):
        k = int(w.outage[b])
        keep = None if k < 0 else np.arange(w.net.n_line) != k
        el, ev = _compare(res, b, nets[b], w.loads[b], kw, 1e-5, 1e-4, keep=keep)
        worst_l, worst_v = max(worst_l, el), max(worst_v, ev)
    print(f"batched {precision} {rule}: worst lambda rel err {worst_l:.2e}, value {worst_v:.2e}")
