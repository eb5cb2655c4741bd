"""GPU parity of dcopf_dual_eval and dcopf_dual_certify_bound against the FP64 oracle.

Tolerances: FP64 products match the oracle's dual value to 1e-9 relative (the
oracle and the GPU sum in different orders; both are FP64), FP32 products and BF16
hi/lo split products on tensor cores to 1e-5 relative with FP64 accumulation.
"Relative" is to |g| + |lambda| D, the size of the Lagrangian's dominant term: at a
random dual point g itself can be a near-total cancellation of terms of that size.  Gradients are compared elementwise, dispatches
per generator; LP points with a near-zero reduced cost (a legitimate tie) are
redrawn."""
import numpy as np
import pytest
import torch

from oracle import dcopf
from paper_2406_13191_gb300 import DcopfDual, synth

from gpu_common import drop_line, near_tie, onet, rand_point

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, (net, base) in {
        "c0": synth.network_for(0),
        "c1": synth.network_for(1),
        "tiny_qp": synth.tiny_network(5, 40, 60, 9, quadratic=True),
        "tiny_lp": synth.tiny_network(6, 37, 55, 7),
    }.items():
        out[name] = (net, base, onet(net), DcopfDual(net))
    return out


def _points(on, loads, rng, n, **kw):
    pts = []
    while len(pts) < n:
        p = rand_point(rng, on.n_line, **kw)
        if not near_tie(on, loads, *p):
            pts.append(p)
    return pts


@pytest.mark.parametrize("name", ["c0", "c1", "tiny_qp", "tiny_lp"])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("fp32", 1e-5), ("bf16x3", 1e-5)])
def test_eval_matches_oracle(cases, name, precision, rtol):
    net, base, on, g = cases[name]
    rng = np.random.default_rng(17)
    B = 3
    loads = synth.scenario_loads(base, B, 99)
    pts = []
    for b in range(B):
        pts += _points(on, loads[b], rng, 1)
    lam = np.array([p[0] for p in pts])
    mh = np.stack([p[1] for p in pts])
    ml = np.stack([p[2] for p in pts])
    r = g.eval(loads, lam, mh, ml, precision=precision)
    torch.cuda.synchronize()
    for b in range(B):
        val, gl, ghi, glo, p = dcopf.evaluate(on, loads[b], lam[b], mh[b], ml[b])
        v = r["value"][b].item()
        assert abs(v - val) <= rtol * (abs(val) + abs(lam[b]) * loads[b].sum()), (v, val)
        fscale = 1.0 + np.max(np.abs(on.fmax))
        gtol = {"fp64": 1e-9, "fp32": 2e-4, "bf16x3": 1e-3}[precision] * fscale
        assert np.max(np.abs(r["g_mu_hi"][b].cpu().numpy() - ghi)) <= gtol
        assert np.max(np.abs(r["g_mu_lo"][b].cpu().numpy() - glo)) <= gtol
        assert abs(r["g_lambda"][b].item() - gl) <= (1e-9 if precision == "fp64" else 1e-4) * (1 + loads[b].sum())
        ptol = {"fp64": 1e-9, "fp32": 1e-4, "bf16x3": 1e-3}[precision]
        assert np.max(np.abs(r["dispatch"][b].cpu().numpy() - p)) <= ptol * (1 + np.max(on.pmax))


def test_eval_outage_matches_rebuilt_network(cases):
    net, base, on, g = cases["tiny_lp"]
    br = g.bridge_mask()
    cand = np.flatnonzero(~br)
    rng = np.random.default_rng(23)
    B = 4
    loads = synth.scenario_loads(base, B, 5)
    outage = np.array([-1, cand[0], cand[len(cand) // 2], cand[-1]], dtype=np.int32)
    pts = [rand_point(rng, on.n_line) for _ in range(B)]
    lam = np.array([p[0] for p in pts])
    mh = np.stack([p[1] for p in pts])
    ml = np.stack([p[2] for p in pts])
    for prec, rtol in (("fp64", 1e-9), ("fp32", 1e-5), ("bf16x3", 1e-5)):
        r = g.eval(loads, lam, mh, ml, outage=outage, precision=prec)
        for b in range(B):
            k = outage[b]
            if k < 0:
                o, mhb, mlb = on, mh[b], ml[b]
            else:
                o = drop_line(net, k)
                keep = np.arange(on.n_line) != k
                mhb, mlb = mh[b][keep], ml[b][keep]
            val, gl, ghi, glo, p = dcopf.evaluate(o, loads[b], lam[b], mhb, mlb)
            assert abs(r["value"][b].item() - val) <= rtol * (abs(val) + abs(lam[b]) * loads[b].sum())
            gh = r["g_mu_hi"][b].cpu().numpy()
            if k >= 0:
                assert gh[k] == 0.0
                gh = gh[np.arange(on.n_line) != k]
            assert np.max(np.abs(gh - ghi)) <= {"fp64": 1e-9, "fp32": 2e-4, "bf16x3": 1e-3}[prec] * (1 + on.fmax.max())


@pytest.mark.parametrize("name", ["c0", "c1", "tiny_qp"])
def test_certify_matches_oracle_and_bounds(cases, name):
    net, base, on, g = cases[name]
    rng = np.random.default_rng(31)
    B = 4
    loads = synth.scenario_loads(base, B, 7)
    pts = [rand_point(rng, on.n_line) for _ in range(B)]
    lam = np.array([p[0] for p in pts])
    mh = np.stack([p[1] for p in pts]) - 50.0   # some negative entries: projected by certify
    ml = np.stack([p[2] for p in pts])
    bound, err = g.certify(loads, lam, mh, ml)
    for b in range(B):
        ref = dcopf.dual_value_prices(on, loads[b], lam[b], np.maximum(mh[b], 0), np.maximum(ml[b], 0))
        e = err[b].item()
        assert 0 < e <= 1e-9 * (1 + abs(ref))
        assert abs(bound[b].item() + e - ref) <= 1e-11 * abs(ref)
        # a lower bound of the value (up to the oracle's own FP64 rounding)
        assert bound[b].item() <= ref + 1e-12 * abs(ref)


def test_certify_outage_matches_rebuilt(cases):
    net, base, on, g = cases["tiny_qp"]
    cand = np.flatnonzero(~g.bridge_mask())
    rng = np.random.default_rng(37)
    loads = synth.scenario_loads(base, 3, 8)
    outage = np.array([cand[1], -1, cand[-2]], dtype=np.int32)
    pts = [rand_point(rng, on.n_line) for _ in range(3)]
    lam = np.array([p[0] for p in pts])
    mh = np.stack([p[1] for p in pts])
    ml = np.stack([p[2] for p in pts])
    bound, err = g.certify(loads, lam, mh, ml, outage=outage)
    for b in range(3):
        k = outage[b]
        keep = np.arange(on.n_line) != k
        o = on if k < 0 else drop_line(net, k)
        ref = dcopf.dual_value_prices(o, loads[b], lam[b], mh[b][keep] if k >= 0 else mh[b],
                                      ml[b][keep] if k >= 0 else ml[b])
        assert abs(bound[b].item() + err[b].item() - ref) <= 1e-10 * abs(ref)
        assert 0 < err[b].item() and bound[b].item() <= ref + 1e-12 * abs(ref)


def test_eval_rejects_bad_outages(cases):
    from paper_2406_13191_gb300._lib import DcopfError
    net, base, on, g = cases["c0"]
    z = np.zeros((1, on.n_line))
    br = np.flatnonzero(g.bridge_mask())
    assert len(br) > 0          # the 30-bus network is tree-like: it has bridges
    with pytest.raises(DcopfError) as e:
        g.eval(base[None], np.zeros(1), z, z, outage=np.array([br[0]], dtype=np.int32))
    assert e.value.code == 2
    for bad in (-2, on.n_line):
        with pytest.raises(DcopfError) as e:
            g.eval(base[None], np.zeros(1), z, z, outage=np.array([bad], dtype=np.int32))
        assert e.value.code == 1


def test_bounded_wait_gives_up_and_device_stays_usable(cases):
    """A device wait on a flag that nothing sets returns DCOPF_ERR_TIMEOUT after its
    limit; afterwards the same handle still evaluates correctly."""
    import ctypes as C
    import time
    net, base, on, g = cases["c0"]
    t0 = time.time()
    code = g.lib.dcopf_selftest_bounded_wait(g.h, 20_000_000, C.c_void_p(0))   # 20 ms
    assert code == 5
    assert time.time() - t0 < 5.0
    assert g.lib.dcopf_dual_device_error(g.h) == 0
    r = g.eval(base[None], [-3000.0], np.zeros((1, on.n_line)), np.zeros((1, on.n_line)))
    ref = dcopf.dual_value_prices(on, base, -3000.0, np.zeros(on.n_line), np.zeros(on.n_line))
    assert abs(r["value"][0].item() - ref) <= 1e-9 * abs(ref)


@pytest.mark.parametrize("cfg,batch", [(2, 4), (3, 2)])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("fp32", 1e-5), ("bf16x3", 1e-5)])
def test_eval_full_size_sampled(cfg, batch, precision, rtol):
    """The 4600-bus (with line outages) and 10000-bus workloads at full size: the first
    instances of each, at seeded dual points, against the oracle (rebuilt network for
    an outage)."""
    w = synth.workload(cfg, batch=batch)
    net = w.net
    on = onet(net)
    g = DcopfDual(net)
    rng = np.random.default_rng(100 + cfg)
    pts = [rand_point(rng, net.n_line, density=0.05) for _ in range(batch)]
    lam = np.array([p[0] for p in pts])
    mh = np.stack([p[1] for p in pts])
    ml = np.stack([p[2] for p in pts])
    out = w.outage if (w.outage >= 0).any() else None
    r = g.eval(w.loads, lam, mh, ml, outage=out, precision=precision)
    for b in range(batch):
        k = w.outage[b]
        if k >= 0:
            o = drop_line(net, k)
            keep = np.arange(net.n_line) != k
            val = dcopf.dual_value_lagrangian(o, w.loads[b], lam[b], mh[b][keep], ml[b][keep])
        else:
            val = dcopf.dual_value_lagrangian(on, w.loads[b], lam[b], mh[b], ml[b])
        scale = abs(val) + abs(lam[b]) * w.loads[b].sum()
        assert abs(r["value"][b].item() - val) <= rtol * scale, (b, r["value"][b].item(), val)
