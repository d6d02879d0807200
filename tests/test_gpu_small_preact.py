"""Parity on a network whose pre-activations are small (|a| of order 1e-2), where
tanh(a) ~ a: the FP32 tanh jet must keep its relative accuracy there (a value of
tanh computed as 1 - 2/(exp(2a) + 1) would carry an absolute error of ~1e-7, a
relative error of ~1e-5 at these sizes).  Every output channel, the residual and
the gradients are held to 1e-5 (normwise) against the oracle, for the paths that
evaluate the tanh jet in FP32 at FP32 accuracy: the FP32 kernels and split-BF16.
(BF16 and TF32 are not tested here: their operand rounding, 2^-9 and 2^-12, is what
sets their error, and on this network the derivative channels are four to ten
orders of magnitude below u, so that the normwise error of u_x and u_xx measures
cancellation, not the tanh.)"""
import numpy as np
import pytest

import synth
from oracle import lrnr64
from tests.gpu_common import as_f32_batch, as_f32_net, eim_for, install_fast, rel

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-5}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def small_case(seed=91, L=3, M=64, r=16):
    g = synth.rng(seed)
    net = synth.make_net(g, L=L, M=M, r=r)
    # scale every hidden layer's bases and biases so that the pre-activations stay
    # near 1e-2 (the input layer keeps (x, t) of order one; the output layer is linear)
    for l in range(L):
        net.U[l] = net.U[l] * (0.05 if l == 0 else 0.3)
        net.b[l] = net.b[l] * 0.03
    net = as_f32_net(net)
    bt = as_f32_batch(synth.make_batch(g, net, [900, 211], [64, 33], [40, 17], [5.0, 2.0],
                                       [1.0, 0.5], [2.0, 1.0]))
    return net, bt


def test_the_case_has_small_preactivations():
    net, bt = small_case()
    s = bt.s[0]
    for l in range(net.L):
        z = lrnr64.hidden_states(net, s, bt.x_int[:200], bt.t_int[:200], l)
        a = np.arctanh(z)
        assert np.median(np.abs(a)) < 0.05, l


@pytest.mark.parametrize("form,prec", [("full", "fp32"), ("fast", "fp32"), ("full", "bf16x3"),
                                       ("fast", "bf16x3")])
def test_small_preactivation_outputs_and_gradient(P, form, prec):
    net, bt = small_case()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    ref = net
    if form == "fast":
        rows, Xis, _ = eim_for(net, bt.s[0], 16)
        install_fast(P, model, rows, Xis)
        ref = lrnr64.make_fast(net, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    tol = TOL[prec]
    out = P.lrnr_residual(model, form, prec, db)
    jets, R, Bic, _ = lrnr64.residual_eval(ref, bt, form)
    for c, k in enumerate(("u", "u_t", "u_x", "u_xx")):
        assert rel(out[k].cpu(), jets[:, c]) < tol, (k, rel(out[k].cpu(), jets[:, c]))
    assert rel(out["res"].cpu(), R) < tol
    assert rel(out["res_ic"].cpu(), Bic) < tol
    lo, ds, dbb = P.lrnr_residual_grad(model, form, prec, db)
    ro, rs, rb = lrnr64.residual_grad(ref, bt, form)
    assert rel(lo.cpu(), ro) < tol
    assert rel(ds.cpu(), rs) < tol, rel(ds.cpu(), rs)
    assert rel(dbb.cpu(), rb) < tol, rel(dbb.cpu(), rb)
    assert P.lrnr_last_device_status(model) == 0
