"""FP64 CPU oracle of the Adam update on the coefficients ``s`` (Sec. 4 uses Adam,
Kingma and Ba 2015) and of the locality-regularised fast loss (Eq. 3.7).

TEST INFRASTRUCTURE ONLY (see ``oracle/lrnr64.py``).

One step at count ``k`` (1-based) for gradient ``g``:
    m <- b1 m + (1 - b1) g
    v <- b2 v + (1 - b2) g^2
    s <- s - lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)
The paper gives no hyper-parameters; defaults b1 = 0.9, b2 = 0.999, eps = 1e-8.
"""
from __future__ import annotations

import numpy as np


def adam_step(s, m, v, k, g, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** k)
    vhat = v / (1.0 - b2 ** k)
    s = s - lr * mhat / (np.sqrt(vhat) + eps)
    return s, m, v


def locality_term(s, anchor, lam):
    """``lam * sum |s - anchor|`` (Eq. 3.7) and its subgradient (sign(0) = 0)."""
    d = s - anchor
    return lam * np.sum(np.abs(d), axis=-1), lam * np.sign(d)


def spinprop_loop(loss_grad, s0, n_steps, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8,
                  lam=0.0, anchor=None):
    """Run ``n_steps`` Adam steps on ``s`` with gradient ``loss_grad(s) -> (loss, g)``
    plus the locality term; returns final s, m, v and the loss of the last step."""
    s = np.array(s0, dtype=np.float64, copy=True)
    m = np.zeros_like(s)
    v = np.zeros_like(s)
    loss = None
    for k in range(1, n_steps + 1):
        loss, g = loss_grad(s)
        if lam and anchor is not None:
            lt, lg = locality_term(s, anchor, lam)
            loss = loss + lt
            g = g + lg
        s, m, v = adam_step(s, m, v, k, g, lr, b1, b2, eps)
    return s, m, v, loss
