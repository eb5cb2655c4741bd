"""Clusters of two CTA pairs in the batched tensor-core products.

Tile codes 5 .. 8 run the pair tiles of codes 1 .. 4 in clusters of two pairs that
compute neighbouring column tiles: each box of the batch operand (H for the adjoint, X
for the forward) is loaded once and multicast to the CTAs of the same rank in both
pairs, and a stage is refilled only when both pairs' MMAs have read it.  Every output
element is still the same sequence of MMAs over the same K blocks, so a solve must be
bit for bit the one with one pair per cluster: a box landing in the wrong CTA or a
stage refilled too early would change the products and so the iterations.
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
QP_ADAM = dict(rule="adam", alpha=3000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000)


def _solve(net, shape, monkeypatch, loads, outage, gam, **kw):
    monkeypatch.setenv("DCOPF_TENSOR_SHAPE", shape)
    g = DcopfDual(net)
    monkeypatch.delenv("DCOPF_TENSOR_SHAPE")
    r = g.solve(loads, outage=outage, target=gam, gap=1e-3, path="batched", precision="bf16x3", **kw)
    torch.cuda.synchronize()
    return g.tensor_shapes(), [t.cpu().numpy().copy() for t in (r.status, r.iters, r.bound, r.lam, r.mu_hi)]


def _same(net, shapes, monkeypatch, loads, outage, gam, **kw):
    (s1, a), (s2, b) = (_solve(net, sh, monkeypatch, loads, outage, gam, **kw) for sh in shapes)
    assert s2["adjoint"].startswith("2 pairs") and s2["forward"].startswith("2 pairs"), s2
    assert not s1["adjoint"].startswith("2 pairs"), s1
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    st, b0 = a[0], a[2]
    assert np.all(b0 <= gam + 1e-9 * np.abs(gam))
    ok = st == 0
    assert np.all((gam[ok] - b0[ok]) / np.abs(gam[ok]) <= 1e-3 + 1e-12)
    print(f"{s2['lines']} lines, {s1['code']} and {s2['code']}: reached {ok.sum()} of {len(gam)}, "
          f"mean iterations {a[1].mean():.1f}")
    return st


def test_two_pair_clusters_qp_10000bus_screened(monkeypatch):
    """256 instances of the 10000-bus QP, screened: the adjoint on 256 x 160 pairs with
    split-K 4 (16 column tiles), the forward on 256 x 160 pairs (63 column tiles, an odd
    count: the cluster of the last one carries a pair past the last line)."""
    gam = np.array(json.load(open(os.path.join(GOLDEN, "c3_gamma.json")))["gamma"], dtype=float)
    w = synth.workload(3, batch=len(gam))
    loads = torch.tensor(w.loads, dtype=torch.float64, device="cuda")
    st = _same(w.net, ("3,4,3,1", "7,4,7,1"), monkeypatch, loads, None, gam, screen=True, **QP_ADAM)
    assert (st == 0).all()


def test_two_pair_clusters_lp_4600bus_300_with_outages(monkeypatch):
    """300 instances of the 4600-bus LP, every other one with a line outage: two row
    tiles of 256 (the second one ragged), the adjoint on 256 x 144 pairs (18 column
    tiles) with split-K 6, the forward on 256 x 192 pairs (38 column tiles)."""
    gl = json.load(open(os.path.join(GOLDEN, "c2_gamma.json")))["gamma"][:300]
    w = synth.workload(2, batch=300)
    ok = np.array([x is not None for x in gl])
    gam = np.array([x for x in gl if x is not None], dtype=float)
    loads = torch.tensor(w.loads[ok], dtype=torch.float64, device="cuda")
    outage = torch.tensor(w.outage[ok], dtype=torch.int32, device="cuda")
    st = _same(w.net, ("4,6,2,1", "8,6,6,1"), monkeypatch, loads, outage, gam, **LP_ADAM)
    assert (st == 0).mean() > 0.95
