"""What the learned warm start gains on the 2000-bus network.

The perceptron is trained on the GPU (the library's own forward, backward and Adam
kernels) on duals that the method itself produces for seeded training scenarios,
then proposes starting points for held-out scenarios.  Both arms solve the same
held-out instances to a certified 0.1 % gap against the oracle's gamma*
(tests/golden/warm_gamma.json): cold start from lambda = mu = 0 with the tuned
Adam settings, warm start from the proposal with a smaller Adam step.  Every bound
must be valid, every instance must reach the gap, and the warm arm must need at most
60 % of the cold arm's iterations on average."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2406_13191_gb300 import DcopfDual, synth, warmstart

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "warm_gamma.json")
COLD = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000)
WARM = dict(rule="adam", alpha=300.0, beta1=0.9, beta2=0.999, decay=0.997, max_iters=4000)
TARGETS = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=1500,
               tol=0.0, path="batched", precision="bf16x3")


def test_learned_warm_start_needs_fewer_iterations():
    net, _ = synth.network_for(1)
    g = DcopfDual(net)
    Xtr = synth.warm_loads("train", 4096)
    Y, _ = warmstart.dual_targets(g, Xtr, **TARGETS)
    m = warmstart.WarmStartMLP(net.n_bus, 1 + net.n_line, 512, max_batch=1024)
    m.set_params(warmstart.init_params(net.n_bus, 512, 1 + net.n_line, 7))
    m.set_normalization(*warmstart.normalization(Xtr, Y.cpu().numpy()))
    losses = warmstart.train(m, torch.as_tensor(Xtr, dtype=torch.float32, device=m.device),
                             Y.contiguous(), 20, batch=512, lr=1e-3, lr_final=1e-5, seed=11)
    assert losses[-1] < 0.5 * losses[0]
    assert m.device_error() == 0

    n = 256
    Xev = synth.warm_loads("heldout", n)
    gam = np.array(json.load(open(GOLD))["gamma"][:n], dtype=float)
    cold = g.solve(Xev, target=gam, path="batched", precision="bf16x3", **COLD)
    warm = g.solve(Xev, target=gam, path="batched", precision="bf16x3", warm=m.warm_start(Xev), **WARM)
    for r in (cold, warm):
        b = r.bound.cpu().numpy()
        assert np.all(r.status.cpu().numpy() == 0)
        assert np.all(b <= gam + 1e-9 * np.abs(gam))
        assert np.all(b >= gam * (1 - 1e-3) - 1e-9 * np.abs(gam))
    it_cold = cold.iters.double().mean().item()
    it_warm = warm.iters.double().mean().item()
    assert it_warm <= 0.6 * it_cold, (it_warm, it_cold)
