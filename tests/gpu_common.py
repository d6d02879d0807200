"""Helpers shared by the GPU parity tests: build the same seeded workload for the
CUDA library and for the FP64 oracle, and compare them."""
from __future__ import annotations

import numpy as np
import torch

import synth
from oracle import eim64, lrnr64

TOL_FP32 = 1e-5     # normwise relative error of each quantity, FP32 path vs FP64 oracle


def rel(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / n) if n > 0 else float(np.linalg.norm(a - b))


def as_f32_batch(bt):
    """Round the batch to FP32 exactly as the device sees it, so both sides use the
    same inputs."""
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return synth.Batch(beta=f(bt.beta), nu=f(bt.nu), rho=f(bt.rho), s=f(bt.s),
                       int_off=bt.int_off, ic_off=bt.ic_off, bc_off=bt.bc_off,
                       x_int=f(bt.x_int), t_int=f(bt.t_int), x_ic=f(bt.x_ic), t_bc=f(bt.t_bc))


def as_f32_net(net):
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return synth.Net(L=net.L, M=net.M, r=net.r, U=[f(u) for u in net.U], V=[f(v) for v in net.V],
                     b=[f(b) for b in net.b])


def eim_for(net, s, rhat, n_per_point=8, seed=77, tol=0.0):
    """Oracle EIM rows / bases of every hidden layer from the standard snapshot design."""
    g = synth.rng(seed)
    xs, ts = synth.snapshot_design(g, n_per_point)
    rows, Xis, Ss = [], [], []
    for l in range(net.L):
        S = lrnr64.hidden_states(net, s, xs, ts, l)
        p, Xi, _ = eim64.eim_greedy(S, rhat, tol)
        rows.append(p)
        Xis.append(Xi)
        Ss.append(S)
    return rows, Xis, Ss


def install_fast(P, model, rows, Xis):
    for l, (p, Xi) in enumerate(zip(rows, Xis)):
        r_in = torch.tensor(np.asarray(p, np.int32), device="cuda")
        X_in = torch.tensor(np.ascontiguousarray(Xi.T), device="cuda")
        P.fastlrnr_select_rows(model, l, rhat=len(p), rows_in=r_in, Xi_in=X_in)


def per_instance_rel(a, b):
    return max(rel(a[i], b[i]) for i in range(b.shape[0]))


def bc_err(got, Bbc, model, bt, form):
    """Error of the periodic residual B = u(0,t) - u(2pi,t).  B is a difference of
    nearly equal values, so its FP32 error is set by the error of its operands:
    measure ||dB|| against ||u(0, t)|| (the operand scale), not against ||B||."""
    fwd = lrnr64.full_forward if form == "full" else lrnr64.fast_forward
    scale = 0.0
    for i in range(bt.n_inst):
        inst = bt.instance(i)
        if len(inst["t_bc"]):
            u0, _ = fwd(model, inst["s"], np.zeros_like(inst["t_bc"]), inst["t_bc"])
            scale += float(np.sum(u0[:, 0] ** 2))
    d = np.linalg.norm(np.asarray(got, np.float64) - Bbc)
    return d / np.sqrt(scale) if scale > 0 else d


def jet_magnitudes(net, s, x, t):
    """Rounding scale of each output jet channel: the forward pass with every sum
    replaced by the root of the sum of its squared terms (sqrt(V^2^T z^2), ...) and
    the jet rules applied to those scales.  The rounding error of a long sum of terms
    of mixed sign grows like eps times this root-sum-square (not like eps times the
    result), so this is the scale against which the error of an ill-conditioned
    channel -- a small result of large cancelling sums, as u_xx is in deep networks
    with these weights -- is measured."""
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    off = np.cumsum([0] + list(net.r))
    Zm = np.zeros((x.shape[0], 4, 2))
    Zm[:, 0, 0], Zm[:, 0, 1] = np.abs(x), np.abs(t)
    Zm[:, 1, 1] = 1.0
    Zm[:, 2, 0] = 1.0
    Zv = lrnr64.input_jets(x, t)
    for l in range(net.L + 1):
        sl = np.asarray(s[off[l]:off[l + 1]], np.float64)
        qm = np.sqrt((Zm ** 2) @ (net.V[l] ** 2)) * np.abs(sl)
        am = np.sqrt((qm ** 2) @ (net.U[l] ** 2).T)
        am[:, 0] = np.sqrt(am[:, 0] ** 2 + net.b[l] ** 2)
        av = ((Zv @ net.V[l]) * sl) @ net.U[l].T
        av[:, 0] += net.b[l]
        if l == net.L:
            return am[:, :, 0]
        z, d1, d2, _ = lrnr64.tanh_derivs(av[:, 0])
        Zv, _ = lrnr64.act_jets(av)
        Zm = np.empty_like(am)
        Zm[:, 0] = np.abs(z)
        Zm[:, 1] = np.abs(d1) * am[:, 1]
        Zm[:, 2] = np.abs(d1) * am[:, 2]
        Zm[:, 3] = np.sqrt((d2 * am[:, 2] ** 2) ** 2 + (d1 * am[:, 3]) ** 2)


def jet_err(got, ref, mag):
    """Normwise error of one jet channel measured against its magnitude."""
    return float(np.linalg.norm(np.asarray(got, np.float64) - ref) / np.linalg.norm(mag))
