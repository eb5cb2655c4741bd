"""Learned warm start: binding of include/dcopf_mlp.h and the training driver.

A perceptron (bus loads -> 512 -> 512 GELU -> (lambda, eta)) proposes the starting
dual point of ``DcopfDual.solve``.  Any proposal with mu >= 0 is a valid dual point
(Section 3, Remarks 1-2), so the network changes only the number of iterations to
the certified gap; cold start stays the fallback.

Every numeric step (forward, loss, backward, Adam, the dual split) runs in
libdcopfdual.so.  This module moves arguments, draws the seeded initial weights and
minibatch orders (random inputs of the method, made on the host), and computes the
per-column normalisation statistics of a data set once on the host.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from .dual import DcopfDual, _as_dev, _ptr


class WarmStartMLP:
    """One perceptron on one GPU (``dcopf_mlp_create``)."""

    def __init__(self, n_in: int, n_out: int, n_hidden: int = 512, max_batch: int = 1024,
                 device: int | None = None, precision: str = "bf16x3"):
        """``precision``: "bf16x3" (products on the tensor cores, BF16 hi/lo split
        operands) or "fp32" (FP32 SIMT products)."""
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            d = _lib.MlpDesc(int(n_in), int(n_hidden), int(n_out), int(max_batch),
                             _lib.PRECISION[precision])
            h = C.c_void_p()
            _lib.check(self.lib.dcopf_mlp_create(C.byref(d), C.byref(h)), "dcopf_mlp_create")
        self.h = h
        self.n_in, self.n_hidden, self.n_out, self.max_batch = n_in, n_hidden, n_out, max_batch
        self.num_params = int(self.lib.dcopf_mlp_num_params(self.h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.dcopf_mlp_destroy(h)
            self.h = None

    def _stream(self):
        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _f32(self, x, shape=None):
        t = _as_dev(x, torch.float32, self.device)
        return t if shape is None else t.reshape(shape)

    def set_params(self, params) -> None:
        p = self._f32(params, (self.num_params,))
        _lib.check(self.lib.dcopf_mlp_set_params(self.h, _ptr(p), self._stream()), "dcopf_mlp_set_params")
        torch.cuda.current_stream(self.device).synchronize()

    def get_params(self) -> torch.Tensor:
        p = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        _lib.check(self.lib.dcopf_mlp_get_params(self.h, _ptr(p), self._stream()), "dcopf_mlp_get_params")
        return p

    def set_normalization(self, in_shift, in_scale, out_shift, out_scale) -> None:
        a = [self._f32(v, (n,)) for v, n in ((in_shift, self.n_in), (in_scale, self.n_in),
                                             (out_shift, self.n_out), (out_scale, self.n_out))]
        _lib.check(self.lib.dcopf_mlp_set_normalization(self.h, *[_ptr(t) for t in a], self._stream()),
                   "dcopf_mlp_set_normalization")
        torch.cuda.current_stream(self.device).synchronize()

    def forward(self, x) -> torch.Tensor:
        x = self._f32(x)
        x = x.reshape(-1, self.n_in)
        y = torch.empty(x.shape[0], self.n_out, dtype=torch.float32, device=self.device)
        _lib.check(self.lib.dcopf_mlp_forward(self.h, x.shape[0], _ptr(x), _ptr(y), self._stream()),
                   "dcopf_mlp_forward")
        return y

    def loss_grad(self, idx, X: torch.Tensor, Y: torch.Tensor):
        idx = _as_dev(idx, torch.int32, self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        grad = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        _lib.check(self.lib.dcopf_mlp_loss_grad(self.h, idx.numel(), _ptr(idx), X.shape[0], _ptr(X),
                                                _ptr(Y), _ptr(loss), _ptr(grad), self._stream()),
                   "dcopf_mlp_loss_grad")
        return loss, grad

    def train_step(self, idx: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, lr: float,
                   beta1=0.9, beta2=0.999, eps=1e-8, loss_out: torch.Tensor | None = None) -> None:
        """One Adam step on rows ``idx`` (int32 CUDA tensor) of X, Y (float32 CUDA)."""
        a = _lib.AdamParams(float(lr), float(beta1), float(beta2), float(eps))
        _lib.check(self.lib.dcopf_mlp_train_step(self.h, idx.numel(), _ptr(idx), X.shape[0], _ptr(X),
                                                 _ptr(Y), C.byref(a), _ptr(loss_out), self._stream()),
                   "dcopf_mlp_train_step")

    def warm_start(self, loads):
        """(lambda [B], mu_hi [B][n_out-1], mu_lo) proposed for loads [B][n_in] (FP64)."""
        L = _as_dev(loads, torch.float64, self.device).reshape(-1, self.n_in)
        B, nl = L.shape[0], self.n_out - 1
        lam = torch.empty(B, dtype=torch.float64, device=self.device)
        mh = torch.empty(B, nl, dtype=torch.float64, device=self.device)
        ml = torch.empty(B, nl, dtype=torch.float64, device=self.device)
        for i in range(0, B, self.max_batch):
            j = min(B, i + self.max_batch)
            _lib.check(self.lib.dcopf_mlp_warm_start(self.h, j - i, _ptr(L[i:j]), _ptr(lam[i:j]),
                                                     _ptr(mh[i:j]), _ptr(ml[i:j]), self._stream()),
                       "dcopf_mlp_warm_start")
        return lam, mh, ml

    def device_error(self) -> int:
        return int(self.lib.dcopf_mlp_device_error(self.h))

    def kernel_launches(self) -> int:
        return int(self.lib.dcopf_mlp_kernel_launches(self.h))


def init_params(n_in: int, n_hidden: int, n_out: int, seed: int) -> np.ndarray:
    """Seeded initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for every weight and
    bias of a layer (flat, in the ABI's parameter order)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_in, fan_out in ((n_in, n_hidden), (n_hidden, n_hidden), (n_hidden, n_out)):
        r = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-r, r, size=fan_in * fan_out))
        parts.append(rng.uniform(-r, r, size=fan_out))
    return np.concatenate(parts).astype(np.float32)


def normalization(X: np.ndarray, Y: np.ndarray, floor: float = 1e-3):
    """Per-column (shift, scale) of inputs (scale = 1/std) and outputs (scale = std),
    with std floored at ``floor`` times the largest column std (constant columns)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    xs = X.std(0)
    xs = np.maximum(xs, floor * max(xs.max(), 1e-30))
    ys = Y.std(0)
    ys = np.maximum(ys, floor * max(ys.max(), 1e-30))
    return (X.mean(0).astype(np.float32), (1.0 / xs).astype(np.float32),
            Y.mean(0).astype(np.float32), ys.astype(np.float32))


def dual_targets(dual: DcopfDual, loads: np.ndarray, chunk: int = 4096, **solve_kw):
    """Training targets from target-free solves of the method (no warm start):
    Y = (lambda, mu_hi - mu_lo) of each instance's best iterate, as float32 rows, and
    the solve status of each row."""
    Ys, st = [], []
    for i in range(0, loads.shape[0], chunk):
        r = dual.solve(loads[i:i + chunk], **solve_kw)
        Ys.append(torch.cat([r.lam[:, None], r.mu_hi - r.mu_lo], 1).float())
        st.append(r.status)
    return torch.cat(Ys), torch.cat(st)


def train(mlp: WarmStartMLP, X: torch.Tensor, Y: torch.Tensor, epochs: int, batch: int = 512,
          lr: float = 1e-3, lr_final: float = 1e-5, seed: int = 0, beta1=0.9, beta2=0.999,
          eps=1e-8) -> list[float]:
    """Minibatch Adam on (X, Y) (float32 CUDA tensors) with a cosine step-size decay
    from ``lr`` to ``lr_final``; returns the mean loss of each epoch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = X.shape[0]
    steps = n // batch
    total = max(1, epochs * steps)
    losses = torch.empty(total, dtype=torch.float32, device=mlp.device)
    out, k = [], 0
    for _ in range(epochs):
        perm = torch.as_tensor(rng.permutation(n)[: steps * batch].astype(np.int32), device=mlp.device)
        k0 = k
        for s in range(steps):
            a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k / total))
            mlp.train_step(perm[s * batch:(s + 1) * batch], X, Y, a, beta1, beta2, eps,
                           loss_out=losses[k:k + 1])
            k += 1
        out.append(float(losses[k0:k].mean().item()))
    return out
