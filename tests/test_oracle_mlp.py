"""Pins of the oracle's warm-start perceptron (oracle/mlp.py) against facts that do
not come from the oracle.

Hand case (tests/golden/mlp_hand.json): one input, one unit per layer.  With x = 1,
W1 = 1, b1 = 0 the first unit is GELU(1) = Phi(1).  W2 = 2, b2 = -2 Phi(1) make the
second pre-activation exactly 0, so GELU gives 0 and u = b3 = 0.25 whatever W3 is.
For target 0 the loss is 0.0625 and, by the chain rule with GELU'(0) = 1/2 and
GELU'(1) = Phi(1) + phi(1):
  dL/db3 = 2u = 0.5,  dL/dW3 = 0.5 * 0 = 0,  dL/db2 = 0.5 * 5 * 1/2 = 1.25,
  dL/dW2 = 1.25 Phi(1),  dL/db1 = 1.25 * 2 * (Phi(1) + phi(1)) = dL/dW1 (x = 1).
"""
import json
import os

import numpy as np
import pytest

from oracle import mlp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mlp_hand.json")))
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def test_gelu_textbook_values():
    Phi1, phi1 = GOLD["Phi1"], GOLD["phi1"]
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(1.0)) - Phi1) < 1e-15
    assert abs(mlp.gelu(np.array(-1.0)) + (1.0 - Phi1)) < 1e-15
    z = np.linspace(-6, 6, 25)
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-14, rtol=0)   # z Phi(z) + z Phi(-z) = z
    assert abs(mlp.gelu_grad(np.array(0.0)) - 0.5) < 1e-15
    assert abs(mlp.gelu_grad(np.array(1.0)) - (Phi1 + phi1)) < 1e-15
    assert mlp.gelu_grad(np.array(40.0)) == 1.0 and mlp.gelu(np.array(40.0)) == 40.0


def test_hand_network_forward_and_gradient():
    p = np.array([GOLD["params"][k] for k in ORDER])
    dims = (1, 1, 1)
    xn = np.array([[GOLD["x"]]])
    z1, h1, z2, h2, u = mlp.forward(p, dims, xn)
    assert abs(h1[0, 0] - GOLD["h1"]) < 1e-15
    assert abs(z2[0, 0] - GOLD["z2"]) < 1e-15
    assert abs(u[0, 0] - GOLD["u"]) < 1e-15
    loss, g = mlp.loss_grad(p, dims, xn, np.array([[GOLD["target"]]]))
    assert abs(loss - GOLD["loss"]) < 1e-15
    for k, gv in zip(ORDER, g):
        assert abs(gv - GOLD["grad"][k]) < 1e-14, k


def test_linear_regime_is_an_affine_map():
    """Pre-activations far above zero make GELU the identity in FP64, so the network
    is the affine map x -> ((x W1 + b1) W2 + b2) W3 + b3; rectangular layers catch a
    transposed weight."""
    rng = np.random.default_rng(3)
    dims = (5, 4, 3)
    W1, W2, W3 = (rng.uniform(0.1, 0.2, s) for s in ((5, 4), (4, 4), (4, 3)))
    b1, b2, b3 = np.full(4, 50.0), np.full(4, 50.0), rng.normal(size=3)
    p = np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)])
    x = rng.uniform(0, 1, (2, 5))
    u = mlp.forward(p, dims, x)[4]
    aff = ((x @ W1 + b1) @ W2 + b2) @ W3 + b3
    assert np.allclose(u, aff, rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_by_central_differences(seed):
    rng = np.random.default_rng(seed)
    dims = (5, 4, 3)
    P = mlp.num_params(*dims)
    p = rng.normal(scale=0.7, size=P)
    xn = rng.normal(size=(3, 5))
    tn = rng.normal(size=(3, 3))
    _, g = mlp.loss_grad(p, dims, xn, tn)
    h = 1e-6
    fd = np.empty(P)
    for i in range(P):
        e = np.zeros(P)
        e[i] = h
        fd[i] = (mlp.loss_grad(p + e, dims, xn, tn)[0] - mlp.loss_grad(p - e, dims, xn, tn)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * (1 + np.max(np.abs(g)))


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient the bias-corrected moments equal g and g^2 exactly, so
    each step moves every parameter by lr g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3])
    p0 = np.array([1.0, 2.0, 3.0])
    p, m, v = p0.copy(), np.zeros(3), np.zeros(3)
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        p, m, v = mlp.adam_step(p, g, m, v, t, lr, 0.9, 0.999, eps)
    assert np.allclose(p, p0 - 5 * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)


def test_to_duals_split():
    lam, mh, ml = mlp.to_duals(np.array([[-7.0, 2.0, -3.0, 0.0]]))
    assert lam[0] == -7.0
    assert mh.tolist() == [[2.0, 0.0, 0.0]] and ml.tolist() == [[0.0, 3.0, 0.0]]
