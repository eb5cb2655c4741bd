"""Eq. (16)'s QP dual with s as an ascent variable (Section 3.2, Remark 2) on the plain
FP64 path, against the oracle's own implementation (oracle/dcopf.py, solve_qp_s, pinned
in tests/test_oracle_pins.py::test_qp_dual_with_s_variable).

The GPU ascends on g_q(lambda, mu, s) with the same rule and schedule; both keep the
point with the largest g_q, and the GPU's certified bound at that point is the
closed-form dual value g(lambda, mu) = max_s g_q, which the oracle reports as
best_closed.  FP64 throughout, so lambda and the bound agree to 1e-8.
"""
import numpy as np
import pytest
import torch

from oracle import dcopf
from paper_2406_13191_gb300 import DcopfDual, _lib, synth

from gpu_common import gamma, onet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    s_, loads = synth.tiny_network(23, 16, 24, 6, quadratic=True)
    return s_, loads, onet(s_), DcopfDual(s_)


@pytest.mark.parametrize("rule,kw", [("adam", dict(alpha=1000.0, beta1=0.9, beta2=0.999, decay=0.998)),
                                     ("gdm", dict(alpha=2.0, alpha_lambda=0.5, rho=0.9, decay=0.99))])
def test_plain_s_ascent_follows_oracle(qp, rule, kw):
    net, loads, on, g = qp
    res = g.solve(loads[None], path="plain", precision="fp64", rule=rule, max_iters=30, qp_dual="s", **kw)
    torch.cuda.synchronize()
    ref = dcopf.solve_qp_s(on, loads, rule=rule, max_iters=30, **kw)
    assert res.iters[0].item() == 30 and res.status[0].item() == 1
    assert abs(res.lam[0].item() - ref["lam"]) <= 1e-8 * max(1.0, abs(ref["lam"]))
    assert abs(res.bound[0].item() - ref["best_closed"]) <= 1e-8 * abs(ref["best_closed"])
    assert np.allclose(res.mu_hi[0].cpu().numpy(), ref["mu_hi"], rtol=1e-8, atol=1e-8)


def test_plain_s_ascent_reaches_gap(qp):
    net, loads, on, g = qp
    gam = gamma(on, loads)
    res = g.solve(loads[None], path="plain", precision="fp64", rule="adam", alpha=1000.0, beta1=0.9,
                  beta2=0.999, decay=0.998, max_iters=5000, target=[gam], qp_dual="s")
    torch.cuda.synchronize()
    b = res.bound[0].item()
    assert res.status[0].item() == 0
    assert gam * (1 - 1e-3) - 1e-9 * abs(gam) <= b <= gam + 1e-9 * abs(gam)


def test_s_ascent_only_on_the_plain_qp_path(qp):
    net, loads, on, g = qp
    for path in ("fused", "batched"):
        with pytest.raises(_lib.DcopfError) as e:
            g.solve(loads[None], path=path, max_iters=5, qp_dual="s")
        assert e.value.code == 6
    lp, lp_loads = synth.tiny_network(6, 37, 55, 7)
    with pytest.raises(_lib.DcopfError) as e:
        DcopfDual(lp).solve(lp_loads[None], path="plain", precision="fp64", max_iters=5, qp_dual="s")
    assert e.value.code == 6
