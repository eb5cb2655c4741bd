"""Randomised parity of the CUDA path against the FP64 oracle: seeded networks of
assorted sizes (LP and QP, with and without line outages), seeded dual points, every
precision of dcopf_dual_eval, and the certificate.

Outage instances are compared with the oracle on the network rebuilt without the
line.  Tolerances as in test_gpu_eval.py: the value to 1e-9 (FP64) or 1e-5 (FP32 and
BF16 hi/lo) of |g| + |lambda| D; the certificate below the oracle's value (up to the
oracle's own rounding) and within its rounding allowance of it."""
import numpy as np
import pytest

from oracle import dcopf
from paper_2406_13191_gb300 import DcopfDual, synth

from gpu_common import drop_line, near_tie, onet, rand_point

pytestmark = pytest.mark.gpu

# (seed, buses, lines, generators, quadratic, instances, outages)
CASES = [(101, 23, 31, 4, False, 5, 2), (102, 57, 80, 13, True, 6, 3),
         (103, 140, 190, 31, True, 7, 3), (104, 96, 150, 9, False, 4, 2),
         (105, 210, 300, 70, True, 9, 4)]


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[1]}" for c in CASES])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("fp32", 1e-5), ("bf16x3", 1e-5)])
def test_random_networks_eval_and_certify(case, precision, rtol):
    seed, nb, nl, ng, qp, B, n_out = case
    w = synth.scenario_workload(seed, nb, nl, ng, qp, batch=B, n_out=n_out)
    on = onet(w.net)
    g = DcopfDual(w.net)
    rng = np.random.default_rng(seed)
    lam, mh, ml, refs = [], [], [], []
    for b in range(B):
        k = int(w.outage[b])
        o = on if k < 0 else drop_line(w.net, k)
        keep = np.arange(nl) != k
        while True:
            p = rand_point(rng, nl)
            if k >= 0:
                p[1][k] = p[2][k] = 0.0   # the outaged line carries no multiplier
            if not near_tie(o, w.loads[b], p[0], p[1][keep], p[2][keep]):
                break
        lam.append(p[0])
        mh.append(p[1])
        ml.append(p[2])
        refs.append((o, keep))
    lam, mh, ml = np.array(lam), np.stack(mh), np.stack(ml)
    r = g.eval(w.loads, lam, mh, ml, outage=w.outage, precision=precision, want_grad=False,
               want_dispatch=False)
    bound, err = g.certify(w.loads, lam, mh, ml, outage=w.outage)
    for b in range(B):
        o, keep = refs[b]
        val = dcopf.dual_value_prices(o, w.loads[b], lam[b], mh[b][keep], ml[b][keep])
        scale = abs(val) + abs(lam[b]) * w.loads[b].sum()
        assert abs(r["value"][b].item() - val) <= rtol * scale, (b, r["value"][b].item(), val)
        if precision == "fp64":
            e = err[b].item()
            assert 0 < e <= 1e-9 * scale
            assert bound[b].item() <= val + 1e-12 * abs(val)
            assert abs(bound[b].item() + e - val) <= 1e-10 * scale
