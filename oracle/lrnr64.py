"""FP64 CPU oracle of the LRNR / FastLRNR physics-informed hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never imports it.

What it computes, in plain FP64 NumPy, point by point (vectorised over points):

* LRNR forward (Sec. 2.1, Eq. 2.1 with Eq. 2.2): hidden layers
  ``z^l = tanh(U^l diag(s^l) V^l^T z^{l-1} + b^l)``, linear last layer, input
  ``z^0 = (x, t)``, scalar output ``u``.  The input derivatives ``u_t, u_x, u_xx``
  are carried forward as Taylor jets (chain rule written out; the paper obtains
  the same exact derivatives by automatic differentiation).
* FastLRNR forward (Sec. 2.2, Eqs. 2.6-2.8): ``zhat^l = Vhat^{l+1 T} tanh(Uhat^l
  (s^l * zhat^{l-1}) + bhat^l)`` with ``zhat^0 = V^{1 T} z^0`` and output
  ``U^{L+1}(s^{L+1} * zhat^L) + b^{L+1}``.
* CDR residual and initial / periodic boundary operators (Sec. 4, Eq. 4.1).
* Losses: mean-square fine-tune loss (Eq. 3.5) and l1 fast loss (Eq. 3.6).
* The exact gradient of the loss with respect to ``s`` and ``b`` (reverse mode
  through the jets, the backpropagation that Sec. 2.3 counts).

Notation: weight layers are indexed ``l = 0..L`` here (the paper's ``1..L+1``);
``L`` is the number of activated (hidden) layers.  Jet channels are ordered
``(value, d/dt, d/dx, d^2/dx^2)``.

Readings of the paper taken here (each is listed with its reason in the design
notes): ``V^l`` has ``M_{l-1}`` rows (the printed ``M_l`` cannot multiply
``z^{l-1}``); the reduced layer keeps the bias, ``bhat = P^T b``; the activation
is ``tanh``; the periodic condition constrains values only; the MSE loss is three
separate means; the l1 loss is plain sums with ``sign(0) = 0``.
"""
from __future__ import annotations

import numpy as np

CH_U, CH_T, CH_X, CH_XX = 0, 1, 2, 3
NCH = 4


# ---------------------------------------------------------------------------
# Activation jets
# ---------------------------------------------------------------------------

def tanh_derivs(a0: np.ndarray):
    """tanh and its first three derivatives at ``a0``."""
    z = np.tanh(a0)
    d1 = 1.0 - z * z
    d2 = -2.0 * z * d1
    d3 = d1 * (6.0 * z * z - 2.0)
    return z, d1, d2, d3


def act_jets(a: np.ndarray):
    """Push the jet ``a[..., c, :]`` through tanh (chain rule, second order in x).

    ``a`` has shape ``(N, 4, m)``.  Returns the output jet and the derivative
    values needed by the adjoint.
    """
    a0, at, ax, axx = a[:, CH_U], a[:, CH_T], a[:, CH_X], a[:, CH_XX]
    z, d1, d2, d3 = tanh_derivs(a0)
    out = np.empty_like(a)
    out[:, CH_U] = z
    out[:, CH_T] = d1 * at
    out[:, CH_X] = d1 * ax
    out[:, CH_XX] = d2 * ax * ax + d1 * axx
    return out, (d1, d2, d3)


def act_jets_adjoint(a: np.ndarray, derivs, zbar: np.ndarray) -> np.ndarray:
    """Adjoint of :func:`act_jets`: given ``zbar`` (same shape), return ``abar``."""
    d1, d2, d3 = derivs
    at, ax, axx = a[:, CH_T], a[:, CH_X], a[:, CH_XX]
    zb0, zbt, zbx, zbxx = zbar[:, CH_U], zbar[:, CH_T], zbar[:, CH_X], zbar[:, CH_XX]
    abar = np.empty_like(a)
    abar[:, CH_U] = (zb0 * d1 + zbt * d2 * at + zbx * d2 * ax
                     + zbxx * (d3 * ax * ax + d2 * axx))
    abar[:, CH_T] = zbt * d1
    abar[:, CH_X] = zbx * d1 + 2.0 * zbxx * d2 * ax
    abar[:, CH_XX] = zbxx * d1
    return abar


def input_jets(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Jet of the input ``z^0 = (x, t)``: value, d/dt = (0,1), d/dx = (1,0), d2/dx2 = 0."""
    n = x.shape[0]
    z = np.zeros((n, NCH, 2))
    z[:, CH_U, 0] = x
    z[:, CH_U, 1] = t
    z[:, CH_T, 1] = 1.0
    z[:, CH_X, 0] = 1.0
    return z


def split_s(s: np.ndarray, r) -> list:
    out, o = [], 0
    for rl in r:
        out.append(np.asarray(s[o:o + rl], dtype=np.float64))
        o += rl
    return out


# ---------------------------------------------------------------------------
# Full LRNR (Eq. 2.1-2.2)
# ---------------------------------------------------------------------------

def full_forward(net, s, x, t):
    """Jets ``u[:, c]`` of the LRNR at points (x, t) and the cache for the adjoint."""
    sl = split_s(s, net.r)
    Z = input_jets(np.asarray(x, np.float64), np.asarray(t, np.float64))
    cache = []
    L = net.L
    for l in range(L + 1):
        q = Z @ net.V[l]                 # (N, 4, r_l):  q_c = V^T z_c
        p = q * sl[l]                    # diag(s) q
        a = p @ net.U[l].T               # (N, 4, M_l):  a_c = U p_c
        a[:, CH_U] += net.b[l]           # bias enters the value channel only
        if l < L:
            Z, derivs = act_jets(a)
            cache.append((q, a, derivs))
        else:
            cache.append((q, a, None))
            u = a[:, :, 0]               # (N, 4) linear output layer
    return u, cache


def full_backward(net, s, cache, ubar):
    """Reverse pass: ``ubar`` (N, 4) -> (dL/ds flat, list of dL/db per layer)."""
    sl = split_s(s, net.r)
    L = net.L
    ds = [None] * (L + 1)
    db = [None] * (L + 1)
    abar = ubar[:, :, None]              # output layer is linear: abar = ubar
    for l in range(L, -1, -1):
        q, a, derivs = cache[l]
        if l < L:
            abar = act_jets_adjoint(a, derivs, zbar)
        db[l] = abar[:, CH_U].sum(axis=0)
        pbar = abar @ net.U[l]           # (N, 4, r_l)
        ds[l] = (pbar * q).sum(axis=(0, 1))
        qbar = pbar * sl[l]
        zbar = qbar @ net.V[l].T         # (N, 4, M_{l-1})
    return np.concatenate(ds), db


# ---------------------------------------------------------------------------
# FastLRNR (Eq. 2.6-2.8)
# ---------------------------------------------------------------------------

class FastNet:
    """Reduced bases: ``Uh[l]`` (rh_l, r_l), ``bh[l]`` (rh_l,), ``Vh[l]`` (rh_l, r_{l+1}),
    plus the row sets ``rows[l]`` for l = 0..L-1, the input ``V[0]`` and output
    ``U[L]``, ``b[L]`` of the full net (trivial reductions at input and output)."""

    def __init__(self, net, rows, Uh, bh, Vh):
        self.net = net
        self.L = net.L
        self.r = net.r
        self.rows = [np.asarray(p, dtype=np.int64) for p in rows]
        self.Uh, self.bh, self.Vh = Uh, bh, Vh


def reduce_layer(U, b, Vnext, rows, Xi):
    """EIM reduction of one activated layer (Eq. 2.7):
    ``Uhat = P^T U``, ``bhat = P^T b``, ``Vhat = (P^T Xi)^{-T} Xi^T V^{l+1}``."""
    rows = np.asarray(rows, dtype=np.int64)
    PtXi = Xi[rows, :]                   # (rh, rh)
    G = Xi.T @ Vnext                     # (rh, r_{l+1})
    Vh = np.linalg.solve(PtXi.T, G)
    return U[rows, :].copy(), b[rows].copy(), Vh


def make_fast(net, rows_list, Xi_list) -> FastNet:
    Uh, bh, Vh = [], [], []
    for l in range(net.L):
        u_, b_, v_ = reduce_layer(net.U[l], net.b[l], net.V[l + 1], rows_list[l], Xi_list[l])
        Uh.append(u_)
        bh.append(b_)
        Vh.append(v_)
    return FastNet(net, rows_list, Uh, bh, Vh)


def fast_forward(fnet, s, x, t):
    net = fnet.net
    sl = split_s(s, net.r)
    L = net.L
    Z0 = input_jets(np.asarray(x, np.float64), np.asarray(t, np.float64))
    zh = Z0 @ net.V[0]                   # zhat^0 = V^{1T} z^0  (N, 4, r_0)
    cache = []
    for l in range(L):
        y = zh * sl[l]
        a = y @ fnet.Uh[l].T             # (N, 4, rh_l)
        a[:, CH_U] += fnet.bh[l]
        w, derivs = act_jets(a)
        cache.append((zh, a, derivs))
        zh = w @ fnet.Vh[l]              # (N, 4, r_{l+1})
    y = zh * sl[L]
    u = (y @ net.U[L].T)[:, :, 0]
    u[:, CH_U] += net.b[L][0]
    cache.append((zh, None, None))
    return u, cache


def fast_backward(fnet, s, cache, ubar):
    """Reverse pass of the FastLRNR; dL/db is scattered to the selected rows."""
    net = fnet.net
    sl = split_s(s, net.r)
    L = net.L
    ds = [None] * (L + 1)
    db = [None] * (L + 1)
    zhL = cache[L][0]
    pbar = ubar[:, :, None] @ net.U[L]   # (N, 4, r_L)
    ds[L] = (pbar * zhL).sum(axis=(0, 1))
    db[L] = np.array([ubar[:, CH_U].sum()])
    zhbar = pbar * sl[L]                 # adjoint of zhat^L
    for l in range(L - 1, -1, -1):
        zh, a, derivs = cache[l]
        wbar = zhbar @ fnet.Vh[l].T      # (N, 4, rh_l)
        abar = act_jets_adjoint(a, derivs, wbar)
        full_db = np.zeros(net.b[l].shape[0])
        np.add.at(full_db, fnet.rows[l], abar[:, CH_U].sum(axis=0))
        db[l] = full_db
        pbar = abar @ fnet.Uh[l]         # (N, 4, r_l)
        ds[l] = (pbar * zh).sum(axis=(0, 1))
        zhbar = pbar * sl[l]
    return np.concatenate(ds), db


# ---------------------------------------------------------------------------
# PDE operators and losses (Eq. 3.5, 3.6, 4.1)
# ---------------------------------------------------------------------------

def cdr_residual(u, ut, ux, uxx, beta, nu, rho):
    """N[u; mu] = u_t + beta u_x - nu u_xx - rho u (1 - u)   (Eq. 4.1)."""
    return ut + beta * ux - nu * uxx - rho * u * (1.0 - u)


def _sign(v):
    return np.sign(v)  # sign(0) = 0


def instance_loss_grad(fwd, bwd, model, inst, loss="mse", w=(1.0, 1.0, 1.0), counts=None):
    """Loss, dL/ds and dL/db of one PDE instance.

    ``fwd``/``bwd`` select the full or the reduced network.  The loss is
    ``w_int mean R^2 + w_ic mean B_ic^2 + w_bc mean B_bc^2`` (MSE, Eq. 3.5) or
    ``w_int sum|R| + w_ic sum|B_ic| + w_bc sum|B_bc|`` (l1, Eq. 3.6).  A term whose
    point set is empty is absent.

    ``counts`` = (N_int, N_ic, N_bc), optional: the MSE terms become
    ``w sum(.^2) / N`` with these denominators instead of the means over the points
    given.  Evaluated on a subset of an instance's points with the whole
    instance's counts, this is that subset's share of the instance's loss and
    gradient: Eq. 3.5's means are sums over the collocation points divided by the
    point counts, and the gradient is a sum over points (Sec. 2.3).
    """
    s = inst["s"]
    beta, nu, rho = inst["beta"], inst["nu"], inst["rho"]
    xi, ti = inst["x_int"], inst["t_int"]
    xc = inst["x_ic"]
    tb = inst["t_bc"]
    ni, nc, nb = xi.shape[0], xc.shape[0], tb.shape[0]
    # one forward over all points: interior, initial (t=0), pairs (0,t) then (2pi,t)
    X = np.concatenate([xi, xc, np.zeros(nb), np.full(nb, 2.0 * np.pi)])
    T = np.concatenate([ti, np.zeros(nc), tb, tb])
    u, cache = fwd(model, s, X, T)
    ubar = np.zeros_like(u)
    total = 0.0
    if ni:
        uu = u[:ni]
        R = cdr_residual(uu[:, CH_U], uu[:, CH_T], uu[:, CH_X], uu[:, CH_XX], beta, nu, rho)
        if loss == "mse" and counts is not None:
            total += w[0] * np.sum(R * R) / counts[0]
            g = 2.0 * w[0] * R / counts[0]
        elif loss == "mse":
            total += w[0] * np.mean(R * R)
            g = 2.0 * w[0] * R / ni
        else:
            total += w[0] * np.sum(np.abs(R))
            g = w[0] * _sign(R)
        ubar[:ni, CH_U] = -rho * (1.0 - 2.0 * uu[:, CH_U]) * g
        ubar[:ni, CH_T] = g
        ubar[:ni, CH_X] = beta * g
        ubar[:ni, CH_XX] = -nu * g
    if nc:
        B = u[ni:ni + nc, CH_U] - np.sin(xc)
        if loss == "mse" and counts is not None:
            total += w[1] * np.sum(B * B) / counts[1]
            ubar[ni:ni + nc, CH_U] = 2.0 * w[1] * B / counts[1]
        elif loss == "mse":
            total += w[1] * np.mean(B * B)
            ubar[ni:ni + nc, CH_U] = 2.0 * w[1] * B / nc
        else:
            total += w[1] * np.sum(np.abs(B))
            ubar[ni:ni + nc, CH_U] = w[1] * _sign(B)
    if nb:
        o = ni + nc
        B = u[o:o + nb, CH_U] - u[o + nb:o + 2 * nb, CH_U]
        if loss == "mse" and counts is not None:
            total += w[2] * np.sum(B * B) / counts[2]
            g = 2.0 * w[2] * B / counts[2]
        elif loss == "mse":
            total += w[2] * np.mean(B * B)
            g = 2.0 * w[2] * B / nb
        else:
            total += w[2] * np.sum(np.abs(B))
            g = w[2] * _sign(B)
        ubar[o:o + nb, CH_U] = g
        ubar[o + nb:o + 2 * nb, CH_U] = -g
    ds, db = bwd(model, s, cache, ubar)
    return float(total), ds, np.concatenate(db)


def residual_grad(model, batch, form="full", loss="mse", w=(1.0, 1.0, 1.0), counts=None):
    """Per-instance loss (n_inst,), dL/ds (n_inst, sum r), dL/db (n_inst, L*M+1).
    ``counts`` (n_inst, 3), optional: each instance's MSE denominators (see
    :func:`instance_loss_grad`)."""
    fwd, bwd = (full_forward, full_backward) if form == "full" else (fast_forward, fast_backward)
    losses, dss, dbs = [], [], []
    for i in range(batch.n_inst):
        ci = None if counts is None else counts[i]
        l_, ds, db = instance_loss_grad(fwd, bwd, model, batch.instance(i), loss, w, ci)
        losses.append(l_)
        dss.append(ds)
        dbs.append(db)
    return np.array(losses), np.stack(dss), np.stack(dbs)


def residual_eval(model, batch, form="full"):
    """Per-point outputs: interior jets (n_int, 4), residual (n_int,), initial and
    periodic boundary residuals."""
    fwd = full_forward if form == "full" else fast_forward
    jets, R, Bic, Bbc = [], [], [], []
    for i in range(batch.n_inst):
        inst = batch.instance(i)
        s = inst["s"]
        u, _ = fwd(model, s, inst["x_int"], inst["t_int"])
        jets.append(u)
        R.append(cdr_residual(u[:, 0], u[:, 1], u[:, 2], u[:, 3], inst["beta"], inst["nu"], inst["rho"]))
        uc, _ = fwd(model, s, inst["x_ic"], np.zeros_like(inst["x_ic"]))
        Bic.append(uc[:, 0] - np.sin(inst["x_ic"]))
        tb = inst["t_bc"]
        u0, _ = fwd(model, s, np.zeros_like(tb), tb)
        u1, _ = fwd(model, s, np.full_like(tb, 2.0 * np.pi), tb)
        Bbc.append(u0[:, 0] - u1[:, 0])
    cat = lambda v, shp: np.concatenate(v) if v else np.zeros(shp)
    return cat(jets, (0, 4)), cat(R, (0,)), cat(Bic, (0,)), cat(Bbc, (0,))


def hidden_states(net, s, x, t, layer):
    """Exact LRNR hidden state ``z^layer = tanh(U s V^T z + b)`` (value channel),
    shape (M, n_points): the snapshots EIM is built from (Sec. 4)."""
    sl = split_s(s, net.r)
    z = np.stack([np.asarray(x, np.float64), np.asarray(t, np.float64)], axis=1)
    for l in range(layer + 1):
        a = ((z @ net.V[l]) * sl[l]) @ net.U[l].T + net.b[l]
        z = np.tanh(a)
    return z.T.copy()
