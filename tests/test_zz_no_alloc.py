"""dcopf_dual_eval_noalloc, called through the C ABI, against dcopf_dual_eval.

The no-allocation variant exists for callers that cannot allocate device memory
themselves: code embedded in a host framework that owns every device allocation,
or a real-time control loop where cudaMalloc's implicit synchronisation and latency
are not acceptable.  It keeps its intermediates in a fixed device array compiled
into the library.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2406_13191_gb300 import DcopfDual, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-5}   # the eval parity tolerances of the other GPU tests
PREC = {"fp64": 0, "fp32": 1}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _call(g, name, loads, outage, lam, mh, ml, prec):
    dev = g.device
    B = loads.shape[0]
    kw = dict(dtype=torch.float64, device=dev)
    out = dict(value=torch.full((B,), np.nan, **kw), g_lambda=torch.full((B,), np.nan, **kw),
               g_mu_hi=torch.full((B, g.n_line), np.nan, **kw),
               g_mu_lo=torch.full((B, g.n_line), np.nan, **kw),
               dispatch=torch.full((B, g.n_gen), np.nan, **kw))
    fn = getattr(g.lib, name)
    code = fn(g.h, B, _ptr(loads), _ptr(outage), _ptr(lam), _ptr(mh), _ptr(ml), PREC[prec],
              _ptr(out["value"]), _ptr(out["g_lambda"]), _ptr(out["g_mu_hi"]),
              _ptr(out["g_mu_lo"]), _ptr(out["dispatch"]),
              C.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    torch.cuda.synchronize(dev)
    return code, out


def _inputs(g, base, B, seed, outage=None):
    rng = np.random.default_rng(seed)
    dev = g.device
    loads = torch.tensor(synth.scenario_loads(base, B, seed), dtype=torch.float64, device=dev)
    lam = torch.tensor(-rng.uniform(1000, 5000, B), dtype=torch.float64, device=dev)
    mask = rng.random((2, B, g.n_line)) < 0.3
    mh = torch.tensor(rng.exponential(300.0, (B, g.n_line)) * mask[0], dtype=torch.float64, device=dev)
    ml = torch.tensor(rng.exponential(300.0, (B, g.n_line)) * mask[1], dtype=torch.float64, device=dev)
    out = None if outage is None else torch.tensor(outage, dtype=torch.int32, device=dev)
    return loads, out, lam, mh, ml


def _compare(a, b, lam, loads, prec):
    tol = TOL[prec]
    scale = a["value"].abs() + lam.abs() * loads.sum(1)
    assert torch.all((a["value"] - b["value"]).abs() <= tol * scale)
    fs = 1.0 + a["g_mu_hi"].abs().max()
    for k in ("g_mu_hi", "g_mu_lo"):
        assert torch.all((a[k] - b[k]).abs() <= tol * 10 * fs)
    assert torch.all((a["g_lambda"] - b["g_lambda"]).abs() <= tol * (1 + loads.sum(1)))
    assert torch.all((a["dispatch"] - b["dispatch"]).abs() <= tol * 10)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_eval_two_calls(prec):
    net, base = synth.network_for(1)
    g = DcopfDual(net)
    for call, (B, seed) in enumerate(((3, 11), (5, 12))):     # two calls in a row
        args = _inputs(g, base, B, seed)
        c1, ref = _call(g, "dcopf_dual_eval", *args, prec)
        c2, got = _call(g, "dcopf_dual_eval_noalloc", *args, prec)
        assert c1 == 0 and c2 == 0, (call, c1, c2)
        _compare(got, ref, args[2], args[0], prec)


def test_noalloc_with_outages_two_calls():
    w = synth.scenario_workload(91, 40, 60, 8, True, batch=6, n_out=3)
    g = DcopfDual(w.net)
    base = w.loads[0]
    for seed in (21, 22):
        loads, _, lam, mh, ml = _inputs(g, base, 6, seed)
        out = torch.tensor(w.outage, dtype=torch.int32, device=g.device)
        c1, ref = _call(g, "dcopf_dual_eval", loads, out, lam, mh, ml, "fp64")
        c2, got = _call(g, "dcopf_dual_eval_noalloc", loads, out, lam, mh, ml, "fp64")
        assert c1 == 0 and c2 == 0
        _compare(got, ref, lam, loads, "fp64")


def test_noalloc_rejects_batches_beyond_the_scratch():
    net, base = synth.network_for(1)
    g = DcopfDual(net)
    # about 111 KB per instance of this network: 1000 instances exceed 16 MiB
    args = _inputs(g, base, 1000, 5)
    code, _ = _call(g, "dcopf_dual_eval_noalloc", *args, "fp64")
    assert code == 1
