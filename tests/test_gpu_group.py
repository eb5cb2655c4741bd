"""dcopf_dual_solve_group: networks of different sizes solved together, each round
one CUDA-graph launch over all of them.  The group must give every network exactly
what its own dcopf_dual_solve_batch gives (same kernels, same inputs, deterministic
reductions); every bound must be valid (at most the oracle's gamma*), and those of
instances that report the target reached within the 0.1 % gap."""
import numpy as np
import pytest
import torch

from paper_2406_13191_gb300 import DcopfDual, _lib, solve_group, synth

from gpu_common import drop_line, gamma, onet

pytestmark = pytest.mark.gpu

ADAM_LP = dict(rule="adam", alpha=1000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=6000)
ADAM_QP = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000)


def _case(seed, nb, nl, ng, qp, B, n_out):
    w = synth.scenario_workload(seed, nb, nl, ng, qp, batch=B, n_out=n_out)
    on = onet(w.net)
    gams = [gamma(on if w.outage[b] < 0 else drop_line(w.net, w.outage[b]), w.loads[b])
            for b in range(B)]
    return w, DcopfDual(w.net), np.array(gams)


@pytest.fixture(scope="module")
def cases():
    return [_case(81, 60, 90, 12, True, 6, 2), _case(82, 37, 55, 7, False, 9, 3),
            _case(83, 120, 170, 20, True, 4, 0)]


def test_group_equals_separate_solves_and_bounds_are_valid(cases):
    kws = [ADAM_QP if w.net.is_qp else ADAM_LP for w, _, _ in cases]
    grp = solve_group([g for _, g, _ in cases], [w.loads for w, _, _ in cases],
                      outage=[w.outage for w, _, _ in cases], target=[t for _, _, t in cases],
                      per_network=kws, precision="bf16x3", path="batched")
    for (w, g, gams), kw, r in zip(cases, kws, grp):
        one = g.solve(w.loads, outage=w.outage, target=gams, path="batched", precision="bf16x3", **kw)
        torch.testing.assert_close(r.iters, one.iters, rtol=0, atol=0)
        torch.testing.assert_close(r.status, one.status, rtol=0, atol=0)
        torch.testing.assert_close(r.bound, one.bound, rtol=0, atol=0)
        torch.testing.assert_close(r.mu_hi, one.mu_hi, rtol=0, atol=0)
        b = r.bound.cpu().numpy()
        st = r.status.cpu().numpy()
        assert np.all(b <= gams + 1e-9 * np.abs(gams))            # every bound is valid
        ok = st == 0                                               # reached the gap
        assert ok.mean() >= 0.75
        assert np.all(b[ok] >= gams[ok] * (1 - 1e-3) - 1e-9 * np.abs(gams[ok]))


def test_group_rejects_repeated_handles_and_other_precisions(cases):
    w, g, gams = cases[0]
    with pytest.raises(_lib.DcopfError) as e:
        solve_group([g, g], [w.loads, w.loads], precision="bf16x3", **ADAM_QP)
    assert e.value.code == 1                     # DCOPF_ERR_INVALID_ARG
    with pytest.raises(_lib.DcopfError) as e:
        solve_group([g], [w.loads], precision="fp32", **ADAM_QP)
    assert e.value.code == 6                     # DCOPF_ERR_UNSUPPORTED


def test_group_mix_300_2000_4600_reaches_stored_optima():
    """The mixed-size workload at full size: 1024 scenarios of the 300-bus QP network,
    256 of the 2000-bus QP network and 128 instances of the 4600-bus LP batch (64 with
    a line outage), one group solve against the oracle's optima
    (tests/golden/group_gamma.json, c2_gamma.json)."""
    import json
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden")
    gg = json.load(open(os.path.join(gold, "group_gamma.json")))
    g2 = json.load(open(os.path.join(gold, "c2_gamma.json")))["gamma"][:128]
    n300, b300 = synth.network_for(300)
    w1 = synth.workload(1, batch=256)
    w2 = synth.workload(2, batch=128)
    assert all(x is not None for x in gg["300"] + gg["2000"] + g2)
    qp = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997)
    lp = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.99, decay=0.99)
    targets = [np.array(gg["300"]), np.array(gg["2000"]), np.array(g2)]
    duals = [DcopfDual(n300), DcopfDual(w1.net), DcopfDual(w2.net)]
    res = solve_group(duals, [synth.scenario_loads(b300, 1024, 4301), w1.loads, w2.loads],
                      outage=[None, None, w2.outage], target=targets, per_network=[qp, qp, lp],
                      max_iters=4000, precision="bf16x3", path="batched", check_every=16)
    torch.cuda.synchronize()
    for r, t in zip(res, targets):
        b = r.bound.cpu().numpy()
        assert (r.status.cpu().numpy() == 0).all()
        assert np.all(b <= t + 1e-9 * np.abs(t)) and np.all(b >= t * (1 - 1e-3) - 1e-9 * np.abs(t))
