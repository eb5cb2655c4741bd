"""FP64 reference of the warm-start perceptron (test infrastructure only).

The paper has no learned component; this is the plain definition of the network
the library trains to propose dual starting points (any dual point with mu >= 0 is
a valid bound, Section 3, Remarks 1-2):

    u = W3^T GELU(W2^T GELU(W1^T xn + b1) + b2) + b3,   GELU(z) = z Phi(z),

with xn = (x - in_shift) * in_scale, targets tn = (y - out_shift) / out_scale, and
the loss L = mean over batch and outputs of (u - tn)^2.  Gradients are the chain
rule written out layer by layer; Adam is Kingma and Ba's bias-corrected update.
Parameters are one flat vector: W1 [n_in][n_h], b1, W2 [n_h][n_h], b2, W3 [n_h][n_out],
b3 (row-major), the layout of the library's ABI.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)


def sizes(n_in: int, nh: int, n_out: int):
    return [(n_in, nh), (nh,), (nh, nh), (nh,), (nh, n_out), (n_out,)]


def num_params(n_in: int, nh: int, n_out: int) -> int:
    return sum(int(np.prod(s)) for s in sizes(n_in, nh, n_out))


def unpack(params, n_in: int, nh: int, n_out: int):
    out, o = [], 0
    for s in sizes(n_in, nh, n_out):
        k = int(np.prod(s))
        out.append(np.asarray(params[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, dims, xn):
    """Layer values for normalised inputs xn [B][n_in]: (z1, h1, z2, h2, u)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, *dims)
    z1 = xn @ W1 + b1
    h1 = gelu(z1)
    z2 = h1 @ W2 + b2
    h2 = gelu(z2)
    u = h2 @ W3 + b3
    return z1, h1, z2, h2, u


def loss_grad(params, dims, xn, tn):
    """Mean squared error against normalised targets tn and its gradient (flat)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, *dims)
    z1, h1, z2, h2, u = forward(params, dims, xn)
    diff = u - tn
    loss = float(np.mean(diff * diff))
    du = 2.0 * diff / diff.size
    gW3 = h2.T @ du
    gb3 = du.sum(0)
    dz2 = (du @ W3.T) * gelu_grad(z2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * gelu_grad(z1)
    gW1 = xn.T @ dz1
    gb1 = dz1.sum(0)
    grad = np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, grad


def adam_step(params, grad, m, v, t, lr, beta1, beta2, eps):
    """Step t (1-based) of bias-corrected Adam; returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def normalise(x, shift, scale):
    return (np.asarray(x, dtype=np.float64) - shift) * scale


def to_duals(y):
    """(lambda, mu_hi, mu_lo) from raw outputs y [B][1 + n_line]."""
    eta = y[:, 1:]
    return y[:, 0], np.maximum(eta, 0.0), np.maximum(-eta, 0.0)
