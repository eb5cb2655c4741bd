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
PREC = {"fp64": 0, "fp32": 1, "bf16x3": 2, 7: 7}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _outputs(g, B):
    kw = dict(dtype=torch.float64, device=g.device)
    return dict(value=torch.full((B,), np.nan, **kw), g_lambda=torch.full((B,), np.nan, **kw),
                g_mu_hi=torch.full((B, g.n_line), np.nan, **kw),
                g_mu_lo=torch.full((B, g.n_line), np.nan, **kw),
                dispatch=torch.full((B, g.n_gen), np.nan, **kw))


def _call(g, name, loads, outage, lam, mh, ml, prec, out=None):
    dev = g.device
    B = loads.shape[0]
    out = _outputs(g, B) if out is None else out
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_with_outages_two_calls(prec):
    w = synth.scenario_workload(91, 40, 60, 8, True, batch=6, n_out=3)
    g = DcopfDual(w.net)
    base = w.loads[0]
    for seed in (21, 22):
        loads, _, lam, mh, ml = _inputs(g, base, 6, seed)
        out = torch.tensor(w.outage, dtype=torch.int32, device=g.device)
        c1, ref = _call(g, "dcopf_dual_eval", loads, out, lam, mh, ml, prec)
        c2, got = _call(g, "dcopf_dual_eval_noalloc", loads, out, lam, mh, ml, prec)
        assert c1 == 0 and c2 == 0
        _compare(got, ref, lam, loads, prec)


def test_noalloc_first_call_on_a_fresh_handle_allocates_nothing():
    """The no-allocation call on a handle that has never allocated a workspace: the
    handle's workspace account stays at zero bytes and the device's free memory does
    not change.  (Another handle makes the first call of the process beforehand, which
    loads the library's device code and with it the fixed array.)"""
    net, base = synth.network_for(1)
    warm = DcopfDual(net)
    args = _inputs(warm, base, 2, 31)
    assert _call(warm, "dcopf_dual_eval_noalloc", *args, "fp64")[0] == 0
    g = DcopfDual(net)
    assert g.workspace_limit() == 0
    for prec in ("fp64", "fp32"):
        args = _inputs(g, base, 4, 32)
        out = _outputs(g, 4)                 # the caller's outputs exist beforehand
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(g.device)[0]
        code, got = _call(g, "dcopf_dual_eval_noalloc", *args, prec, out=out)
        free1 = torch.cuda.mem_get_info(g.device)[0]
        assert code == 0
        assert free1 == free0, (prec, free0 - free1)
        assert g.workspace_limit() == 0
        assert torch.isfinite(got["value"]).all()
    # the allocating call on the same handle then gives the same results
    c1, ref = _call(g, "dcopf_dual_eval", *args, "fp32")
    assert c1 == 0 and g.workspace_limit() > 0
    _compare(got, ref, args[2], args[0], "fp32")


def test_noalloc_batch_above_the_outage_chunk():
    """1500 instances with outages on a small network: the outage indices are checked
    on the host in chunks of 1024, and the scratch still holds the batch."""
    w = synth.scenario_workload(93, 40, 60, 8, False, batch=1500, n_out=600)
    g = DcopfDual(w.net)
    loads, _, lam, mh, ml = _inputs(g, w.loads[0], 1500, 41)
    out = torch.tensor(w.outage, dtype=torch.int32, device=g.device)
    for prec in ("fp64", "fp32"):
        c1, ref = _call(g, "dcopf_dual_eval", loads, out, lam, mh, ml, prec)
        c2, got = _call(g, "dcopf_dual_eval_noalloc", loads, out, lam, mh, ml, prec)
        assert c1 == 0 and c2 == 0
        _compare(got, ref, lam, loads, prec)
    bad = out.clone()
    bad[1200] = w.net.n_line          # out of range, in the second chunk
    c3, _ = _call(g, "dcopf_dual_eval_noalloc", loads, bad, lam, mh, ml, "fp64")
    assert c3 == 1
    c4, _ = _call(g, "dcopf_dual_eval_noalloc", loads, out, lam, mh, ml, "fp64")
    assert c4 == 0   # the rejected call left no error behind


def test_noalloc_precision_codes():
    net, base = synth.network_for(0)
    g = DcopfDual(net)
    args = _inputs(g, base, 2, 51)
    assert _call(g, "dcopf_dual_eval_noalloc", *args, "bf16x3")[0] == 6   # UNSUPPORTED
    assert _call(g, "dcopf_dual_eval_noalloc", *args, 7)[0] == 1          # INVALID_ARG


def test_noalloc_rejects_batches_beyond_the_scratch():
    net, base = synth.network_for(1)
    g = DcopfDual(net)
    # about 111 KB per instance of this network: 1000 instances exceed 16 MiB
    args = _inputs(g, base, 1000, 5)
    code, _ = _call(g, "dcopf_dual_eval_noalloc", *args, "fp64")
    assert code == 1
