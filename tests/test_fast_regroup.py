"""The reduced-coordinate form of the FastLRNR (Eq. 2.8 with the rank-r product
regrouped per layer) against the oracle's rank-coordinate evaluation, in FP64 on the
CPU.  This is the algebra the high-rank FP32 kernel carries out:

  a^0 = K^0 z^0 + bhat^0,      K^0 = Uhat^0 diag(s^0) V^0^T
  a^l = K^l w^{l-1} + bhat^l,  K^l = Uhat^l diag(s^l) Vhat^{l-1 T}
  u   = k w^{L-1} + b^L,       k   = U^L diag(s^L) Vhat^{L-1 T}

and, for the gradient, dL/ds^l_k = sum_ij Uhat^l_ik V_jk G^l_ij with G^l the sum over
points and jet channels of abar^l (outer) w^{l-1} (V = V^0 or Vhat^{l-1}), and
dL/ds^L_k = U^L_k sum_j Vhat^{L-1}_jk g_j with g the sum of ubar_c w^{L-1}_c.  Only the
order of the sums differs from the oracle, so the two agree to rounding."""
import numpy as np
import pytest

import synth
from oracle import eim64 as E
from oracle import lrnr64 as O
from tests.oracle_helpers import relerr


def regrouped_forward(fnet, s, x, t):
    net = fnet.net
    sl = O.split_s(s, net.r)
    L = net.L
    w = O.input_jets(np.asarray(x, np.float64), np.asarray(t, np.float64))
    Ks, keep = [], []
    for l in range(L):
        V = net.V[0] if l == 0 else fnet.Vh[l - 1]
        K = (fnet.Uh[l] * sl[l]) @ V.T
        a = w @ K.T
        a[:, 0] += fnet.bh[l]
        wn, derivs = O.act_jets(a)
        Ks.append(K)
        keep.append((w, a, derivs))
        w = wn
    k = (net.U[L] * sl[L]) @ fnet.Vh[L - 1].T          # (1, rhat_{L-1})
    u = (w @ k.T)[:, :, 0]
    u[:, 0] += net.b[L][0]
    return u, (Ks, k, keep, w)


def regrouped_ds(fnet, s, cache, ubar):
    net = fnet.net
    L = net.L
    Ks, k, keep, wL = cache
    g = np.einsum("nc,ncj->j", ubar, wL)
    ds = [None] * (L + 1)
    ds[L] = net.U[L][0] * (fnet.Vh[L - 1].T @ g)
    wbar = ubar[:, :, None] * k[0]                     # (N, 4, rhat_{L-1})
    for l in range(L - 1, -1, -1):
        w_in, a, derivs = keep[l]
        abar = O.act_jets_adjoint(a, derivs, wbar)
        G = np.einsum("nci,ncj->ij", abar, w_in)
        V = net.V[0] if l == 0 else fnet.Vh[l - 1]
        ds[l] = np.einsum("ik,jk,ij->k", fnet.Uh[l], V, G)
        wbar = abar @ Ks[l]
    return np.concatenate(ds)


@pytest.mark.parametrize("rk,rhat", [((2, 9, 7, 6, 1), 4), ((2, 12, 5, 1), 6), ((1, 8, 1), 3)])
def test_regrouped_fastlrnr_matches_rank_coordinates(rk, rhat):
    g = synth.rng(sum(rk) * 7 + rhat)
    net = synth.make_net_ranks(g, 24, rk)
    s = np.concatenate([g.uniform(0.5, 1.5, r) for r in net.r])
    xs, ts = synth.snapshot_design(g, 4)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _ = E.eim_greedy(O.hidden_states(net, s, xs, ts, l), rhat, 0.0)
        rows.append(p)
        Xis.append(Xi)
    fnet = O.make_fast(net, rows, Xis)
    x, t = g.uniform(0, 2 * np.pi, 50), g.uniform(0, 1, 50)
    u_ref, cache_ref = O.fast_forward(fnet, s, x, t)
    u_rg, cache_rg = regrouped_forward(fnet, s, x, t)
    assert relerr(u_rg, u_ref) < 1e-12
    ubar = g.standard_normal(u_ref.shape)
    ds_ref, _ = O.fast_backward(fnet, s, cache_ref, ubar)
    ds_rg = regrouped_ds(fnet, s, cache_rg, ubar)
    assert relerr(ds_rg, ds_ref) < 1e-11
    assert np.all(np.abs(ds_ref) > 0)                  # every entry carries signal
