"""Edge and degenerate cases of the CUDA path.

- The hand-solved 2-bus and 3-bus networks (tests/golden/hand_cases.json): the dual
  value at the hand-derived dual point is gamma* (eq. (6) at an optimum), its
  certificate is a valid bound just below it, and every solve path reaches it.
- Batch sizes: an empty batch is an argument error, one whose state would not fit the
  32-bit index space is refused before any device access.
- Primal infeasibility (demand above the total capacity): the dual is unbounded, and
  the solve reports it (status 2) once a certified bound exceeds the cost of any
  dispatch (weak duality, Remarks 1-2).
"""
import ctypes as C
import json
import os

import numpy as np
import pytest
import torch

from paper_2406_13191_gb300 import DcopfDual, _lib, synth
from paper_2406_13191_gb300.dual import SolveResult

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))


def hand(name):
    d = GOLD[name]
    net = dict(n_bus=d["n_bus"], line_from=np.array(d["line_from"], np.int32),
               line_to=np.array(d["line_to"], np.int32), line_b=np.array(d["line_b"], float),
               flow_max=np.array(d["flow_max"], float), flow_min=None,
               gen_bus=np.array(d["gen_bus"], np.int32), pmin=np.array(d["pmin"], float),
               pmax=np.array(d["pmax"], float), cost_lin=np.array(d["cost_lin"], float),
               cost_quad=None, base_mva=1.0, slack_bus=0)
    return net, np.array(d["loads"], float), d


@pytest.mark.parametrize("name", ["two_bus", "three_bus"])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_hand_dual_point_gives_gamma(name, precision, rtol):
    net, loads, d = hand(name)
    g = DcopfDual(net)
    lam, mh, ml = [d["lambda"]], [d["mu_hi"]], [d["mu_lo"]]
    r = g.eval(loads[None], lam, mh, ml, precision=precision)
    assert abs(r["value"][0].item() - d["gamma"]) <= rtol * abs(d["gamma"])
    bound, err = g.certify(loads[None], lam, mh, ml)
    assert d["gamma"] - 1e-9 * abs(d["gamma"]) <= bound[0].item() <= d["gamma"]
    assert err[0].item() > 0


@pytest.mark.parametrize("name", ["two_bus", "three_bus"])
@pytest.mark.parametrize("path,precision", [("plain", "fp64"), ("fused", "fp32"),
                                            ("batched", "fp32"), ("batched", "bf16x3")])
def test_hand_solve_reaches_gamma(name, path, precision):
    net, loads, d = hand(name)
    g = DcopfDual(net)
    gam = d["gamma"]
    r = g.solve(loads[None], target=[gam], path=path, precision=precision, rule="adam", alpha=1.0,
                beta1=0.9, beta2=0.999, decay=0.99, max_iters=5000)
    assert r.status[0].item() == 0
    assert gam * (1 - 1e-3) - 1e-9 <= r.bound[0].item() <= gam


def test_batch_size_limits():
    net, base = synth.network_for(0)
    g = DcopfDual(net)
    dev = torch.device("cuda", 0)
    loads = torch.tensor(base[None], device=dev)
    lam = torch.zeros(1, dtype=torch.float64, device=dev)
    mu = torch.zeros(1, net.n_line, dtype=torch.float64, device=dev)
    val = torch.empty(1, dtype=torch.float64, device=dev)
    p = lambda t: C.c_void_p(t.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = g.lib.dcopf_dual_eval(g.h, 0, p(loads), None, p(lam), p(mu), p(mu), 0, p(val), None, None,
                               None, None, s)
    assert rc == 1                              # DCOPF_ERR_INVALID_ARG: empty batch
    huge = (1 << 31) // net.n_line + 1          # batch * n_line beyond 2^31: refused up front
    rc = g.lib.dcopf_dual_eval(g.h, huge, p(loads), None, p(lam), p(mu), p(mu), 0, p(val), None,
                               None, None, None, s)
    assert rc == 6                              # DCOPF_ERR_UNSUPPORTED
    assert g.lib.dcopf_dual_device_error(g.h) == 0


@pytest.mark.parametrize("path", ["plain", "fused", "batched"])
def test_infeasible_instance_is_reported(path):
    net, base = synth.network_for(0)
    g = DcopfDual(net)
    loads = base[None] * (2.0 * net.pmax.sum() / base.sum())   # demand = 2 x total capacity
    prec = {"plain": "fp64", "fused": "fp32", "batched": "bf16x3"}[path]
    r = g.solve(loads, path=path, precision=prec, rule="adam", alpha=1000.0, beta1=0.9, beta2=0.999,
                max_iters=400)
    assert r.status[0].item() == 2
    # the bound itself is still a valid (finite) certified value of the dual
    assert np.isfinite(r.bound[0].item())


@pytest.mark.parametrize("scales", [(1.0, 0.9), (1.0, 0.9, 1.05)])
def test_packed_host_results_equal_the_tensors(scales):
    """One-copy read-back of results that are views of one device buffer (even and odd
    batches: the int32 counts share FP64 slots), and the packing of separate tensors."""
    net, base = synth.network_for(0)
    g = DcopfDual(net)
    loads = np.stack([base * s for s in scales])
    kw = dict(path="batched", precision="bf16x3", rule="adam", alpha=1000.0, beta1=0.95,
              beta2=0.999, decay=0.997, max_iters=50)
    r = g.solve(loads, **kw)
    out = g.new_result(len(scales))
    r2 = g.solve(loads, out=out, **kw)
    assert r2 is out and r.flat is not None
    loose = SolveResult(*(getattr(r, f).clone() for f in ("lam", "mu_hi", "mu_lo", "bound", "iters",
                                                          "status")))
    for res in (r, r2, loose):
        h = res.to_host()
        for f in ("lam", "mu_hi", "mu_lo", "bound", "iters", "status"):
            a, b = getattr(res, f).cpu(), getattr(h, f)
            assert a.shape == b.shape and a.dtype == b.dtype and torch.equal(a, b), f
    # into a reused pinned host result: the same values, twice in a row
    hp = g.new_host_result(len(scales))
    assert hp.flat.is_pinned()
    for res in (r, r2):
        h = res.to_host(into=hp)
        assert h is hp
        for f in ("lam", "mu_hi", "mu_lo", "bound", "iters", "status"):
            a, b = getattr(res, f).cpu(), getattr(h, f)
            assert a.shape == b.shape and a.dtype == b.dtype and torch.equal(a, b), f
    with pytest.raises(ValueError):
        r.to_host(into=g.new_host_result(len(scales) + 1))
    with pytest.raises(ValueError):
        loose.to_host(into=hp)
