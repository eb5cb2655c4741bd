"""Instance groups of the batched tensor-core solve.

A batch can run as two groups whose iteration chains are parallel branches of the
iteration graph, each kernel reading a view of the per-instance state advanced to its
group's first instance.  An instance's arithmetic does not depend on the rows it shares
a product tile with (each output element of an MMA is its own dot product; the split-K
slices, the step's chunks and the minimiser's block size are the same), so with the
product shapes fixed each instance must take exactly the iterations it takes in the
batch run as one group, and end at the same bound.  A wrong offset in any view would
mix instances up and fail that at once.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2406_13191_gb300 import DcopfDual, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LP_ADAM = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.99, decay=0.99, max_iters=1500)
QP_ADAM = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000)


def _handle(net, shape):
    """A handle whose batched products use the fixed shape code "adj,splits,fwd,groups"
    (read when the handle is created)."""
    old = os.environ.get("DCOPF_TENSOR_SHAPE")
    os.environ["DCOPF_TENSOR_SHAPE"] = shape
    try:
        return DcopfDual(net)
    finally:
        if old is None:
            del os.environ["DCOPF_TENSOR_SHAPE"]
        else:
            os.environ["DCOPF_TENSOR_SHAPE"] = old


def _compare(net, loads, outage, gam, shapes, **kw):
    out = []
    for shape in shapes:
        g = _handle(net, shape)
        r = g.solve(loads, outage=outage, target=gam, gap=1e-3, path="batched", precision="bf16x3", **kw)
        torch.cuda.synchronize()
        out.append((g.tensor_shapes(), r.status.cpu().numpy(), r.iters.cpu().numpy(),
                    r.bound.cpu().numpy(), r.lam.cpu().numpy()))
    (s1, st1, it1, b1, l1), (s2, st2, it2, b2, l2) = out
    assert s1["branches"] == 1 and s2["branches"] == 2, (s1, s2)
    assert 0 < s2["first_group"] < len(gam)
    print(f"groups {s2['first_group']} + {len(gam) - s2['first_group']}: "
          f"max |bound diff| / |bound| = {np.max(np.abs(b1 - b2) / np.abs(b1)):.3e}, "
          f"mean iterations {it1.mean():.1f} / {it2.mean():.1f}")
    np.testing.assert_array_equal(st1, st2)
    np.testing.assert_array_equal(it1, it2)
    np.testing.assert_allclose(b2, b1, rtol=1e-12, atol=0)
    np.testing.assert_allclose(l2, l1, rtol=1e-12, atol=0)
    # and every bound is a valid lower bound that reached the gap where it says so
    assert np.all(b2 <= gam + 1e-9 * np.abs(gam))
    assert np.all((gam - b2[st2 == 0]) / np.abs(gam[st2 == 0]) <= 1e-3 + 1e-12)
    return st2


def test_two_groups_match_one_lp_with_outages():
    """300 instances of the 4600-bus LP, every other one with a line outage: groups of 256
    and 43 (a ragged second group in one partial 128-row tile), single-CTA products."""
    gl = json.load(open(os.path.join(GOLDEN, "c2_gamma.json")))["gamma"][:300]
    w = synth.workload(2, batch=300)
    ok = np.array([x is not None for x in gl])
    gam = np.array([x for x in gl if x is not None], dtype=float)
    loads = torch.tensor(w.loads[ok], dtype=torch.float64, device="cuda")
    outage = torch.tensor(w.outage[ok], dtype=torch.int32, device="cuda")
    st = _compare(w.net, loads, outage, gam, ("0,4,0,1", "0,4,0,2"), **LP_ADAM)
    assert (st == 0).mean() > 0.95


def test_two_groups_match_one_qp_screened():
    """256 instances of the 2000-bus QP with constraint screening: two groups of 128."""
    gg = json.load(open(os.path.join(GOLDEN, "group_gamma.json")))
    w = synth.workload(1, batch=256)
    gam = np.array(gg["2000"], dtype=float)
    loads = torch.tensor(w.loads, dtype=torch.float64, device="cuda")
    st = _compare(w.net, loads, None, gam, ("0,3,0,1", "0,3,0,2"), screen=True, **QP_ADAM)
    assert (st == 0).all()


def test_kernel_timing_samples_every_round():
    """The per-kernel timing events of the iteration graph (two event sets, one per round
    parity, so that the host can read a round's while the next one runs): one sample per
    round after the first, positive product and step times."""
    gg = json.load(open(os.path.join(GOLDEN, "group_gamma.json")))
    w = synth.workload(1, batch=256)
    gam = np.array(gg["2000"], dtype=float)
    for shape in ("0,3,0,1", "0,3,0,2"):
        g = _handle(w.net, shape)
        g.set_timing(True)
        g.read_timing()
        g.read_kernel_timing()
        r = g.solve(w.loads, target=gam, gap=1e-3, path="batched", precision="bf16x3", **QP_ADAM)
        torch.cuda.synchronize()
        ms, samples = g.read_kernel_timing()
        it_ms, launches, evals = g.read_timing()
        rounds = -(-int(r.iters.max().item()) // 16)
        print(shape, samples, {k: round(v / max(1, samples) * 1e3, 1) for k, v in ms.items()}, it_ms)
        assert samples >= rounds - 1
        assert ms["adjoint"] > 0 and ms["forward"] > 0 and ms["step"] > 0 and ms["minimiser"] > 0
        assert it_ms > 0 and evals == int(r.iters.sum().item())


def test_iteration_graph_reused_only_for_the_same_arguments():
    """A handle keeps the iteration graph of its last batched solve and replays it for a
    solve whose kernel arguments are the same bytes.  Solves with settings A, B, A on one
    handle: the second A solve (a replay) equals the first bit for bit, and the B solve
    (captured anew) equals B on a fresh handle."""
    gg = json.load(open(os.path.join(GOLDEN, "group_gamma.json")))
    w = synth.workload(1, batch=256)
    gam = np.array(gg["2000"], dtype=float)
    kw_a = dict(QP_ADAM)
    kw_b = dict(QP_ADAM, alpha=2000.0, beta1=0.9)

    def run(g, kw):
        r = g.solve(w.loads, target=gam, gap=1e-3, path="batched", precision="bf16x3", **kw)
        torch.cuda.synchronize()
        return [t.cpu().numpy().copy() for t in (r.bound, r.iters, r.lam, r.mu_hi)]

    g = _handle(w.net, "0,3,0,1")
    a1, b1, a2 = run(g, kw_a), run(g, kw_b), run(g, kw_a)
    fresh = run(_handle(w.net, "0,3,0,1"), kw_b)
    for x, y in zip(a1, a2):
        np.testing.assert_array_equal(x, y)
    for x, y in zip(b1, fresh):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a1[1], b1[1])   # the settings differ in iterations taken


def test_iteration_graph_recaptured_for_another_iteration_cap():
    """The iteration cap is an argument of the graph's kernels (the stop tests): solves
    capped at 40 and then 72 iterations on one handle, with no target, take exactly 40
    and 72 iterations."""
    w = synth.workload(1, batch=256)
    g = _handle(w.net, "0,3,0,1")
    for cap in (40, 72, 40):
        r = g.solve(w.loads, path="batched", precision="bf16x3", **dict(QP_ADAM, max_iters=cap))
        torch.cuda.synchronize()
        it = r.iters.cpu().numpy()
        assert np.all(it == cap), (cap, np.unique(it))
