"""Pin of the oracle's Adam step against torch.optim.Adam (FP64), and the locality term."""
import numpy as np
import torch

import synth
from oracle import adam64 as A


def test_adam_matches_torch_optim():
    g = synth.rng(5)
    s0 = g.uniform(0.5, 1.5, size=17)
    grads = [g.normal(size=17) for _ in range(25)]
    p = torch.tensor(s0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.8, 0.99), eps=1e-7)
    s, m, v = s0.copy(), np.zeros(17), np.zeros(17)
    for k, gk in enumerate(grads, start=1):
        opt.zero_grad()
        p.grad = torch.tensor(gk, dtype=torch.float64)
        opt.step()
        s, m, v = A.adam_step(s, m, v, k, gk, lr=3e-3, b1=0.8, b2=0.99, eps=1e-7)
    assert np.max(np.abs(s - p.detach().numpy())) < 1e-14


def test_locality_term_and_subgradient():
    s = np.array([1.0, 2.0, 3.0, 4.0])
    a = np.array([1.5, 2.0, 2.0, 5.0])
    val, sub = A.locality_term(s, a, 0.25)
    assert val == 0.25 * (0.5 + 0.0 + 1.0 + 1.0)
    assert sub.tolist() == [-0.25, 0.0, 0.25, -0.25]


def test_spinprop_loop_reduces_a_quadratic():
    target = np.array([0.3, -0.7, 1.1])
    f = lambda s: (float(np.sum((s - target) ** 2)), 2 * (s - target))
    s, _, _, loss = A.spinprop_loop(f, np.zeros(3), 400, lr=1e-2)
    assert loss < 1e-3
