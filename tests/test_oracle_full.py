"""Pins of the FP64 oracle's full LRNR path against mathematics, not against itself."""
import math

import numpy as np
import pytest

import synth
from oracle import lrnr64 as O
from tests.oracle_helpers import dense_jets, dense_loss_grad, relerr


def small_case(seed=7, L=3, M=12, r=4, r1=None, n_int=40, n_ic=9, n_bc=6, mu=(5.0, 1.0, 2.0)):
    g = synth.rng(seed)
    net = synth.make_net(g, L=L, M=M, r=r, r1=r1)
    bt = synth.make_batch(g, net, n_int, n_ic, n_bc, *mu)
    return net, bt


def u_value(net, s, x, t):
    u, _ = O.full_forward(net, s, x, t)
    return u[:, 0]


def test_jets_match_central_differences():
    net, bt = small_case()
    s = bt.s[0]
    x, t = bt.x_int, bt.t_int
    u, _ = O.full_forward(net, s, x, t)
    h = 1e-6
    fx = (u_value(net, s, x + h, t) - u_value(net, s, x - h, t)) / (2 * h)
    ft = (u_value(net, s, x, t + h) - u_value(net, s, x, t - h)) / (2 * h)
    # u_xx is small at these weights, so rounding (eps |u| / h^2) dominates at small h:
    # take h = 1e-2 and cancel the h^2 truncation term by Richardson extrapolation.
    d2 = lambda h2: (u_value(net, s, x + h2, t) - 2 * u_value(net, s, x, t)
                     + u_value(net, s, x - h2, t)) / h2**2
    fxx = (4 * d2(5e-3) - d2(1e-2)) / 3
    assert relerr(u[:, 2], fx) < 1e-7
    assert relerr(u[:, 1], ft) < 1e-7
    assert relerr(u[:, 3], fxx) < 1e-6     # rounding ~eps|u|/h^2 over |u_xx| ~ 1e-5


def test_jets_match_dense_autograd():
    net, bt = small_case(seed=11, L=4, M=10, r=3)
    s = bt.s[0]
    u, _ = O.full_forward(net, s, bt.x_int, bt.t_int)
    du, dut, dux, duxx, _, _ = dense_jets(net, s, bt.x_int, bt.t_int)
    for c, ref in enumerate([du, dut, dux, duxx]):
        assert relerr(u[:, c], ref.detach().numpy()) < 1e-13, c


@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_gradient_matches_dense_autograd(loss):
    net, bt = small_case(seed=3)
    inst = bt.instance(0)
    lo, ds, db = O.instance_loss_grad(O.full_forward, O.full_backward, net, inst, loss, (1.0, 0.7, 1.3))
    lr, dsr, dbr = dense_loss_grad(net, inst, loss, (1.0, 0.7, 1.3))
    assert abs(lo - lr) <= 1e-13 * abs(lr)
    assert relerr(ds, dsr) < 1e-12
    assert relerr(db, dbr) < 1e-12


def test_gradient_matches_central_differences_in_s_and_b():
    net, bt = small_case(seed=5, L=3, M=8, r=3, n_int=25, n_ic=7, n_bc=5)
    inst = bt.instance(0)
    lo, ds, db = O.instance_loss_grad(O.full_forward, O.full_backward, net, inst)
    h = 1e-6

    def loss_at(s=None, b=None):
        i2 = dict(inst)
        if s is not None:
            i2["s"] = s
        n2 = net
        if b is not None:
            n2 = synth.Net(L=net.L, M=net.M, r=net.r, U=net.U, V=net.V, b=b)
        return O.instance_loss_grad(O.full_forward, O.full_backward, n2, i2)[0]

    fd_s = np.zeros_like(ds)
    for k in range(ds.shape[0]):
        sp, sm = inst["s"].copy(), inst["s"].copy()
        sp[k] += h
        sm[k] -= h
        fd_s[k] = (loss_at(s=sp) - loss_at(s=sm)) / (2 * h)
    assert relerr(ds, fd_s) < 1e-7
    # biases, layer by layer
    flat = np.concatenate(net.b)
    fd_b = np.zeros_like(flat)
    sizes = [b.shape[0] for b in net.b]
    for k in range(flat.shape[0]):
        fp, fm = flat.copy(), flat.copy()
        fp[k] += h
        fm[k] -= h
        split = lambda f: list(np.split(f, np.cumsum(sizes)[:-1]))
        fd_b[k] = (loss_at(b=split(fp)) - loss_at(b=split(fm))) / (2 * h)
    assert relerr(db, fd_b) < 1e-7


@pytest.mark.parametrize("case", ["travelling", "diffusive", "logistic"])
def test_cdr_residual_closed_forms(case):
    g = synth.rng(1)
    x = g.uniform(0, 2 * math.pi, 50)
    t = g.uniform(0, 1, 50)
    if case == "travelling":     # u = h(x - beta t), nu = rho = 0, h = sin(.) + 0.3 cos(2.)
        beta, nu, rho = 6.5, 0.0, 0.0
        xi = x - beta * t
        hp = np.cos(xi) - 0.6 * np.sin(2 * xi)
        u = np.sin(xi) + 0.3 * np.cos(2 * xi)
        ux, ut, uxx = hp, -beta * hp, -np.sin(xi) - 1.2 * np.cos(2 * xi)
    elif case == "diffusive":    # u = exp(-nu t) sin(x - beta t), rho = 0
        beta, nu, rho = 3.0, 1.7, 0.0
        e = np.exp(-nu * t)
        u = e * np.sin(x - beta * t)
        ux = e * np.cos(x - beta * t)
        uxx = -u
        ut = -nu * u - beta * ux
    else:                        # logistic u(t), beta = nu = 0
        beta, nu, rho = 0.0, 0.0, 2.5
        u0 = 0.2
        u = 1.0 / (1.0 + (1.0 / u0 - 1.0) * np.exp(-rho * t))
        ut = rho * u * (1 - u)
        ux = uxx = np.zeros_like(u)
    R = O.cdr_residual(u, ut, ux, uxx, beta, nu, rho)
    assert np.max(np.abs(R)) < 1e-13


def test_network_of_x_minus_beta_t_has_zero_convection_residual():
    """With r_1 = 1 and V^1 proportional to (1, -beta), the LRNR is a function of
    x - beta t, so u_t + beta u_x = 0 for any downstream weights."""
    beta = 5.0
    net, bt = small_case(seed=21, L=3, M=16, r=5, r1=1, mu=(beta, 0.0, 0.0))
    net.V[0] = np.array([[0.8], [-0.8 * beta]])
    u, _ = O.full_forward(net, bt.s[0], bt.x_int, bt.t_int)
    R = O.cdr_residual(u[:, 0], u[:, 1], u[:, 2], u[:, 3], beta, 0.0, 0.0)
    assert np.max(np.abs(R)) < 1e-12 * max(1.0, np.max(np.abs(u[:, 2])) * beta)
    assert np.max(np.abs(u[:, 2])) > 1e-4   # non-trivial


def test_planted_mistakes_are_caught():
    """A dropped term or a wrong sign in the jet rules fails the autograd pin."""
    net, bt = small_case(seed=2)
    s = bt.s[0]
    du, dut, dux, duxx, _, _ = dense_jets(net, s, bt.x_int, bt.t_int)
    good = O.act_jets

    def bad_jets(a):
        out, d = good(a)
        out[:, O.CH_XX] = d[0] * a[:, O.CH_XX]      # drop sigma'' a_x^2
        return out, d

    O.act_jets = bad_jets
    try:
        u, _ = O.full_forward(net, s, bt.x_int, bt.t_int)
    finally:
        O.act_jets = good
    assert relerr(u[:, 3], duxx.detach().numpy()) > 1e-3
