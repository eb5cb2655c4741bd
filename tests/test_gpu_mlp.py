"""GPU parity of the warm-start perceptron's kernels (include/dcopf_mlp.h) against the
FP64 oracle (oracle/mlp.py), in both modes: FP32 SIMT products, and tcgen05 tensor-core
products with BF16 hi/lo split operands.

Tolerances.  FP32 (FP32 accumulation over K <= 3201 terms): outputs to 2e-5 of the
output scale, each gradient block to 2e-4 of its largest entry, the loss to 1e-5
relative.  BF16 hi/lo (each operand carried to about 2^-16 relative, three products,
FP32 accumulation): ten times wider, outputs 2e-4, gradients 2e-3, loss 1e-4.  Sizes:
the full 2000 -> 512 -> 512 -> 3201 network with a ragged batch of 37 rows (several
tiles and a tail in every dimension, K of the weight gradients a partial tile), and a
small 70 -> 33 -> 129 network for multi-step Adam."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2406_13191_gb300 import warmstart

pytestmark = pytest.mark.gpu

FULL = (2000, 512, 3201)
SMALL = (70, 33, 129)


TOL = {"fp32": dict(out=2e-5, grad=2e-4, loss=1e-5, adam=0.02),
       "bf16x3": dict(out=2e-4, grad=2e-3, loss=1e-4, adam=0.05)}
MODES = ["fp32", "bf16x3"]


def _setup(dims, B, seed, rows=None, precision="fp32"):
    n_in, nh, n_out = dims
    rng = np.random.default_rng(seed)
    rows = rows or B
    X = rng.uniform(0.0, 2.0, (rows, n_in)).astype(np.float32)
    Y = rng.normal(0.0, 3.0, (rows, n_out)).astype(np.float32)
    Y[:, 0] -= 3000.0
    nrm = warmstart.normalization(X, Y)
    p = warmstart.init_params(n_in, nh, n_out, seed)
    m = warmstart.WarmStartMLP(n_in, n_out, nh, max_batch=max(B, 8), precision=precision)
    m.set_params(p)
    m.set_normalization(*nrm)
    return m, X, Y, nrm, p.astype(np.float64)


def _oracle_inputs(X, Y, nrm, idx):
    xs, xsc, ys, ysc = (a.astype(np.float64) for a in nrm)
    xn = omlp.normalise(X[idx], xs, xsc)
    tn = (Y[idx].astype(np.float64) - ys) / ysc
    return xn, tn


@pytest.mark.parametrize("precision", MODES)
@pytest.mark.parametrize("dims,B", [(FULL, 37), (SMALL, 5)])
def test_forward_matches_oracle(dims, B, precision):
    m, X, Y, nrm, p = _setup(dims, B, 1, precision=precision)
    y = m.forward(torch.as_tensor(X, device="cuda")).cpu().numpy().astype(np.float64)
    xn, _ = _oracle_inputs(X, Y, nrm, np.arange(B))
    u = omlp.forward(p, dims, xn)[4]
    ref = nrm[2].astype(np.float64) + nrm[3].astype(np.float64) * u
    scale = nrm[3].astype(np.float64) * (1.0 + np.abs(u).max())
    t = TOL[precision]["out"]
    assert np.all(np.abs(y - ref) <= t * scale[None, :] + t / 20 * np.abs(ref))


@pytest.mark.parametrize("precision", MODES)
@pytest.mark.parametrize("dims,B", [(FULL, 37), (SMALL, 5)])
def test_loss_and_gradient_match_oracle(dims, B, precision):
    rows = 3 * B
    m, X, Y, nrm, p = _setup(dims, B, 2, rows=rows, precision=precision)
    idx = np.random.default_rng(5).choice(rows, B, replace=False).astype(np.int32)
    Xd = torch.as_tensor(X, device="cuda")
    Yd = torch.as_tensor(Y, device="cuda")
    loss, grad = m.loss_grad(idx, Xd, Yd)
    xn, tn = _oracle_inputs(X, Y, nrm, idx)
    lo, go = omlp.loss_grad(p, dims, xn, tn)
    assert abs(loss.item() - lo) <= TOL[precision]["loss"] * lo
    g = grad.cpu().numpy().astype(np.float64)
    o = 0
    for s in omlp.sizes(*dims):
        k = int(np.prod(s))
        ref = go[o:o + k]
        assert np.max(np.abs(g[o:o + k] - ref)) <= TOL[precision]["grad"] * np.max(np.abs(ref)), s
        o += k
    assert m.device_error() == 0


@pytest.mark.parametrize("precision", MODES)
def test_adam_steps_match_oracle(precision):
    dims, B = SMALL, 16
    rows = 64
    m, X, Y, nrm, p = _setup(dims, B, 3, rows=rows, precision=precision)
    Xd = torch.as_tensor(X, device="cuda")
    Yd = torch.as_tensor(Y, device="cuda")
    rng = np.random.default_rng(9)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    po, mo, vo = p.copy(), np.zeros_like(p), np.zeros_like(p)
    g_first = None
    losses = torch.empty(3, dtype=torch.float32, device="cuda")
    for t in range(1, 4):
        idx = rng.choice(rows, B, replace=False).astype(np.int32)
        m.train_step(torch.as_tensor(idx, device="cuda"), Xd, Yd, lr, b1, b2, eps,
                     loss_out=losses[t - 1:t])
        xn, tn = _oracle_inputs(X, Y, nrm, idx)
        lo, go = omlp.loss_grad(po, dims, xn, tn)
        assert abs(losses[t - 1].item() - lo) <= TOL[precision]["loss"] * lo
        if g_first is None:
            g_first = go
        po, mo, vo = omlp.adam_step(po, go, mo, vo, t, lr, b1, b2, eps)
    pg = m.get_params().cpu().numpy().astype(np.float64)
    d = np.abs(pg - po)
    # Adam divides by |g|: entries whose gradient is far above FP32 noise follow the
    # oracle closely; the others can differ by at most the step bound (3 lr).
    big = np.abs(g_first) > 1e-3 * np.abs(g_first).max()
    assert np.max(d[big]) <= TOL[precision]["adam"] * lr
    assert np.max(d) <= 3.0 * lr * 1.01


@pytest.mark.parametrize("precision", MODES)
def test_warm_start_split_matches_forward(precision):
    dims, B = SMALL, 6
    m, X, Y, nrm, p = _setup(dims, B, 4, precision=precision)
    loads = X[:B].astype(np.float64)
    lam, mh, ml = m.warm_start(loads)
    y = m.forward(torch.as_tensor(X[:B], device="cuda")).double()
    torch.testing.assert_close(lam, y[:, 0], rtol=1e-6, atol=1e-6 * y[:, 0].abs().max().item())
    eta = y[:, 1:]
    tol = 1e-6 * (1.0 + eta.abs().max().item())
    assert torch.all(mh >= 0) and torch.all(ml >= 0) and torch.all((mh == 0) | (ml == 0))
    assert torch.max(torch.abs((mh - ml) - eta)).item() <= tol


def test_out_of_range_rows_are_reported():
    dims, B = SMALL, 4
    m, X, Y, nrm, p = _setup(dims, B, 5)
    Xd = torch.as_tensor(X, device="cuda")
    Yd = torch.as_tensor(Y, device="cuda")
    bad = torch.tensor([0, 1, B, 2], dtype=torch.int32, device="cuda")   # B is past the end
    m.loss_grad(bad, Xd, Yd)
    assert m.device_error() == 1            # DCOPF_ERR_INVALID_ARG
    m.loss_grad(torch.tensor([0, 1, 2, 3], dtype=torch.int32, device="cuda"), Xd, Yd)
    assert m.device_error() == 0
