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
