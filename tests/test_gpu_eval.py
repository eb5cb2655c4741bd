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
        scale = abs(val) + abs(lam[b]) * loads[b].sum()
        assert abs(v - val) <= rtol * scale, (v, val)
        if precision == "fp64":
            # FP64 also to 1e-9 of |g| itself (plus the last bits of the summed terms)
            assert abs(v - val) <= 1e-9 * abs(val) + 1e-14 * scale, (v, val)
        print(f"{name} {precision} b={b}: value err {abs(v - val) / abs(val):.2e} of |g|, "
              f"{abs(v - val) / scale:.2e} of |g|+|lambda|D")
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


@pytest.mark.parametrize("cfg", [2, 3])
def test_sparse_certificate_full_size_matches_oracle(cfg):
    """The sparse certificate (level-scheduled LDL^T sweeps, batches above eight or with
    outages) on the 4600-bus network with line outages and on the 10000-bus network,
    twelve instances each: bound + err equals the oracle's FP64 price-form value of the
    projected point (on the network rebuilt without an outaged line), err is small and
    the bound is below the value."""
    w = synth.workload(cfg, batch=12)
    net = w.net
    on = onet(net)
    g = DcopfDual(net)
    rng = np.random.default_rng(41 + cfg)
    pts = [rand_point(rng, net.n_line, density=0.1) for _ in range(w.batch)]
    lam = np.array([p[0] for p in pts])
    mh = np.stack([p[1] for p in pts]) - 20.0   # some negative entries: projected by certify
    ml = np.stack([p[2] for p in pts])
    outage = w.outage if (w.outage >= 0).any() else None
    bound, err = g.certify(w.loads, lam, mh, ml, outage=outage)
    for b in range(w.batch):
        k = int(outage[b]) if outage is not None else -1
        keep = np.arange(net.n_line) != k
        o = on if k < 0 else drop_line(net, k)
        ref = dcopf.dual_value_prices(o, w.loads[b], lam[b], np.maximum(mh[b], 0)[keep],
                                      np.maximum(ml[b], 0)[keep])
        e = err[b].item()
        assert 0 < e <= 1e-9 * (1 + abs(ref)), (b, e)
        assert abs(bound[b].item() + e - ref) <= 1e-10 * abs(ref), (b, bound[b].item() + e, ref)
        assert bound[b].item() <= ref + 1e-12 * abs(ref), b


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


def _safe_point(rng, on, phi_abs, loads, tie_rel):
    """A seeded dual point whose LP reduced costs all stay clear of zero by more than
    tie_rel times the size of their terms (c_j S, lambda, sum_i |Phi_ij| |eta_i|): a
    reduced-precision adjoint cannot flip a generator between its box ends there."""
    while True:
        lam, mh, ml = rand_point(rng, on.n_line, density=0.05)
        if on.qp:
            return lam, mh, ml
        _, _, nu, _, _ = dcopf.dual_parts(on, loads, lam, mh, ml)
        w = on.c * on.S + nu[on.gen_bus]
        size = np.abs(on.c * on.S) + abs(lam) + phi_abs.T @ np.abs(mh - ml)
        if np.all(np.abs(w) > tie_rel * size):
            return lam, mh, ml


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_eval_4600bus_b300_elementwise(precision):
    """300 instances of the 4600-bus LP batch (150 with a line outage): three 128-row
    tiles of the tensor path with a ragged last one, the split-K factor a solve of this
    batch size tuned.  Eight instances spread over the tiles are compared with the
    oracle on the network rebuilt without the outaged line: the dual value, every
    supergradient entry and every generator's dispatch."""
    w = synth.workload(2, batch=300)
    net = w.net
    on = onet(net)
    g = DcopfDual(net)
    if precision == "bf16x3":   # tunes the adjoint's split-K factor for B = 300
        g.solve(w.loads, outage=w.outage, path="batched", precision="bf16x3", max_iters=20)
    sample = [0, 1, 127, 128, 200, 255, 256, 299]
    rng = np.random.default_rng(300)
    nets = {b: (on if w.outage[b] < 0 else drop_line(net, int(w.outage[b]))) for b in sample}
    pts = [rand_point(rng, net.n_line, density=0.05) for _ in range(w.batch)]
    tie_rel = 1e-6 if precision == "fp32" else 1e-4
    for b in sample:
        o = nets[b]
        mask = np.arange(net.n_line) != w.outage[b] if w.outage[b] >= 0 else slice(None)
        phi_abs = np.abs(o.ptdf_gen())
        lam, mh, ml = _safe_point(rng, o, phi_abs, w.loads[b], tie_rel)
        full_h, full_l = np.zeros(net.n_line), np.zeros(net.n_line)
        full_h[mask], full_l[mask] = mh, ml
        pts[b] = (lam, full_h, full_l)
    lam = np.array([p[0] for p in pts])
    mh = np.stack([p[1] for p in pts])
    ml = np.stack([p[2] for p in pts])
    r = g.eval(w.loads, lam, mh, ml, outage=w.outage, precision=precision)
    torch.cuda.synchronize()
    rtol = 1e-5
    gtol = {"fp32": 2e-4, "bf16x3": 1e-3}[precision] * (1.0 + np.max(np.abs(net.flow_max)))
    worst_g = worst_s = worst_grad = worst_p = 0.0
    for b in sample:
        k = int(w.outage[b])
        keep = np.arange(net.n_line) != k
        mhb, mlb = (mh[b][keep], ml[b][keep]) if k >= 0 else (mh[b], ml[b])
        val, gl, ghi, glo, p = dcopf.evaluate(nets[b], w.loads[b], lam[b], mhb, mlb)
        v = r["value"][b].item()
        scale = abs(val) + abs(lam[b]) * w.loads[b].sum()
        worst_g = max(worst_g, abs(v - val) / abs(val))
        worst_s = max(worst_s, abs(v - val) / scale)
        assert abs(v - val) <= rtol * scale, (b, v, val)
        gh = r["g_mu_hi"][b].cpu().numpy()
        go = r["g_mu_lo"][b].cpu().numpy()
        if k >= 0:
            assert gh[k] == 0.0 and go[k] == 0.0
            gh, go = gh[keep], go[keep]
        e = max(np.max(np.abs(gh - ghi)), np.max(np.abs(go - glo)))
        worst_grad = max(worst_grad, e)
        assert e <= gtol, (b, e)
        assert abs(r["g_lambda"][b].item() - gl) <= 1e-4 * (1 + w.loads[b].sum())
        ep = np.max(np.abs(r["dispatch"][b].cpu().numpy() - p))
        worst_p = max(worst_p, ep)
        assert ep <= 1e-9 * (1 + np.max(net.pmax)), (b, ep)   # LP: box ends, exact
    print(f"4600-bus B=300 {precision}: value err {worst_g:.2e} of |g|, {worst_s:.2e} of "
          f"|g|+|lambda|D; gradient {worst_grad:.2e} p.u.; dispatch {worst_p:.1e}")
