"""Independent FP64 cross-checks used to pin the oracle (CPU only).

``dense_*`` evaluates the LRNR as the dense network of Eq. 2.1 with the weight
``W^l = U^l diag(s^l) V^l^T`` formed explicitly, and differentiates it with
torch.autograd; nothing here is shared with ``oracle/``.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64)


def dense_params(net, s):
    """Torch leaves: per-layer s and b, plus constant U, V."""
    off = np.cumsum([0] + list(net.r))
    s_t = [_t(s[off[l]:off[l + 1]]).requires_grad_(True) for l in range(net.L + 1)]
    b_t = [_t(net.b[l]).requires_grad_(True) for l in range(net.L + 1)]
    return s_t, b_t


def dense_u(net, s_t, b_t, X, T):
    z = torch.stack([X, T], dim=-1)
    for l in range(net.L + 1):
        W = _t(net.U[l]) @ torch.diag(s_t[l]) @ _t(net.V[l]).T
        a = z @ W.T + b_t[l]
        z = torch.tanh(a) if l < net.L else a
    return z[:, 0]


def dense_jets(net, s, x, t):
    """u, u_t, u_x, u_xx by autograd (each point's u depends only on its own x, t)."""
    s_t, b_t = dense_params(net, s)
    X = _t(x).requires_grad_(True)
    T = _t(t).requires_grad_(True)
    u = dense_u(net, s_t, b_t, X, T)
    ux, ut = torch.autograd.grad(u.sum(), (X, T), create_graph=True)
    uxx, = torch.autograd.grad(ux.sum(), X, create_graph=True)
    return u, ut, ux, uxx, s_t, b_t


def dense_loss_grad(net, inst, loss="mse", w=(1.0, 1.0, 1.0)):
    """Loss of one instance and its gradient in s (flat) and b (flat), by autograd."""
    beta, nu, rho = inst["beta"], inst["nu"], inst["rho"]
    s_t, b_t = dense_params(net, inst["s"])
    terms = []
    if len(inst["x_int"]):
        X = _t(inst["x_int"]).requires_grad_(True)
        T = _t(inst["t_int"]).requires_grad_(True)
        u = dense_u(net, s_t, b_t, X, T)
        ux, ut = torch.autograd.grad(u.sum(), (X, T), create_graph=True)
        uxx, = torch.autograd.grad(ux.sum(), X, create_graph=True)
        R = ut + beta * ux - nu * uxx - rho * u * (1 - u)
        terms.append(w[0] * ((R * R).mean() if loss == "mse" else R.abs().sum()))
    if len(inst["x_ic"]):
        xc = _t(inst["x_ic"])
        B = dense_u(net, s_t, b_t, xc, torch.zeros_like(xc)) - torch.sin(xc)
        terms.append(w[1] * ((B * B).mean() if loss == "mse" else B.abs().sum()))
    if len(inst["t_bc"]):
        tb = _t(inst["t_bc"])
        B = (dense_u(net, s_t, b_t, torch.zeros_like(tb), tb)
             - dense_u(net, s_t, b_t, torch.full_like(tb, 2 * math.pi), tb))
        terms.append(w[2] * ((B * B).mean() if loss == "mse" else B.abs().sum()))
    Ltot = sum(terms)
    gs = torch.autograd.grad(Ltot, s_t + b_t)
    ds = torch.cat(gs[:net.L + 1]).numpy()
    db = torch.cat(gs[net.L + 1:]).numpy()
    return float(Ltot.detach()), ds, db


def relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(b.ravel())
    return d / n if n > 0 else d
