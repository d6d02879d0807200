"""FastLRNR in FP32 for ranks above the rank-r jet kernel (padded rank 32 or 64, such as
the paper's convection-diffusion-reaction network r = (1, 49, 30, 25, 1)): the
reduced-coordinate kernel (maps K^l = Uhat^l diag(s^l) Vhat^{l-1 T} per tile, the
gradient in s through the tile's rhat x rhat sums) against the FP64 oracle's FastLRNR,
which works in the rank coordinates of Eq. 2.8."""
import numpy as np
import pytest
import torch

import synth
from oracle import adam64, lrnr64
from tests.gpu_common import TOL_FP32, as_f32_batch, as_f32_net, bc_err, eim_for, install_fast, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def case(seed, M, rk, rhat, n_int, n_ic, n_bc, mu):
    g = synth.rng(seed)
    net = as_f32_net(synth.make_net_ranks(g, M, rk))
    k = len(n_int)
    bt = as_f32_batch(synth.make_batch(g, net, n_int, n_ic, n_bc, *[np.full(k, v) for v in mu]))
    rows, Xis, _ = eim_for(net, bt.s[0], rhat)
    return net, bt, rows, Xis


@pytest.mark.parametrize("rk,rhat", [((1, 49, 30, 25, 1), 5), ((1, 20, 24, 1), 12),
                                     ((1, 40, 33, 1), 16)])
@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_high_rank_fastlrnr_gradient_matches_oracle(P, rk, rhat, loss):
    net, bt, rows, Xis = case(sum(rk) + rhat, 96, rk, rhat, [900, 0, 300], [64, 5, 0],
                              [33, 0, 9], (2.0, 1.0, 1.0))
    fnet = lrnr64.make_fast(net, rows, Xis)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db, loss=loss)
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast", loss=loss)
    for i in range(bt.n_inst):
        if ro[i] == 0.0:
            assert lo[i].item() == 0.0 and torch.all(ds[i] == 0)
            continue
        assert abs(lo[i].item() - ro[i]) <= TOL_FP32 * abs(ro[i]), i
        assert rel(ds[i].cpu(), rs[i]) < TOL_FP32, (i, rel(ds[i].cpu(), rs[i]))
        assert rel(dbb[i].cpu(), rb[i]) < TOL_FP32, (i, rel(dbb[i].cpu(), rb[i]))
    assert np.all(dbb.cpu().numpy()[rb == 0.0] == 0.0)       # rows outside P get nothing
    assert P.lrnr_last_device_status(model) == 0


def test_high_rank_fastlrnr_forward_outputs(P):
    net, bt, rows, Xis = case(7, 80, (1, 49, 30, 25, 1), 5, [500], [40], [20], (2.0, 1.0, 1.0))
    fnet = lrnr64.make_fast(net, rows, Xis)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    out = P.lrnr_residual(model, "fast", "fp32", P.DeviceBatch.from_host(bt))
    jets, R, Bic, Bbc = lrnr64.residual_eval(fnet, bt, "fast")
    for c, k in enumerate(("u", "u_t", "u_x", "u_xx")):
        assert rel(out[k].cpu(), jets[:, c]) < TOL_FP32, k
    assert rel(out["res"].cpu(), R) < TOL_FP32
    assert rel(out["res_ic"].cpu(), Bic) < TOL_FP32
    assert bc_err(out["res_bc"].cpu(), Bbc, fnet, bt, "fast") < TOL_FP32


def test_high_rank_spinprop_matches_oracle_adam(P):
    """The paper's fast phase setting on its CDR ranks: Adam steps of the l1 loss plus
    the locality term through the reduced network, FP32, against the oracle's loop."""
    net, bt, rows, Xis = case(11, 64, (1, 49, 30, 25, 1), 5, [12, 30], [0, 4], [0, 2],
                              (2.0, 1.0, 1.0))
    fnet = lrnr64.make_fast(net, rows, Xis)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    s = torch.tensor(bt.s, dtype=torch.float32, device="cuda")
    anchor = s.clone()
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo = torch.zeros(bt.n_inst, dtype=torch.float32, device="cuda")
    n, lr, lam = 5, 1e-2, 1e-3
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, n_steps=n, lr=lr, lambda_loc=lam,
                    s_anchor=anchor, loss="l1", loss_out=lo)
    assert step.item() == n
    for i in range(bt.n_inst):
        inst = bt.instance(i)

        def lg(sv, inst=inst):
            d = dict(inst)
            d["s"] = sv
            l_, g_, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet,
                                                  d, loss="l1")
            return l_, g_
        sr, _, _, lr_ = adam64.spinprop_loop(lg, inst["s"], n, lr=lr, lam=lam, anchor=inst["s"])
        disp = np.abs(sr - inst["s"]).max()
        assert np.max(np.abs(s[i].cpu().numpy() - sr)) <= 1e-2 * disp + 1e-6, i
        assert abs(lo[i].item() - lr_) <= 1e-4 * abs(lr_) + 1e-6, i
    assert P.lrnr_last_device_status(model) == 0


@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_high_rank_fastlrnr_beyond_one_grid_round(P, loss):
    """More tiles than two CTAs per SM: the tile kernel writes per-tile partial rows and a
    separate fixed-order reduction follows (small batches reduce inside the kernel)."""
    n_int = [12000, 9000, 12000, 11000]
    net, bt, rows, Xis = case(5, 96, (1, 49, 30, 25, 1), 5, n_int, [64, 0, 40, 10],
                              [33, 9, 0, 20], (2.0, 1.0, 1.0))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = sum(-(-a // 128) + -(-b // 128) + -(-c // 64)
                for a, b, c in zip(n_int, [64, 0, 40, 10], [33, 9, 0, 20]))
    assert tiles > 2 * sms
    fnet = lrnr64.make_fast(net, rows, Xis)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", P.DeviceBatch.from_host(bt), loss=loss)
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast", loss=loss)
    for i in range(bt.n_inst):
        assert abs(lo[i].item() - ro[i]) <= TOL_FP32 * abs(ro[i]), i
        assert rel(ds[i].cpu(), rs[i]) < TOL_FP32, (i, rel(ds[i].cpu(), rs[i]))
        assert rel(dbb[i].cpu(), rb[i]) < TOL_FP32, (i, rel(dbb[i].cpu(), rb[i]))
    assert P.lrnr_last_device_status(model) == 0


def test_high_rank_fastlrnr_empty_instance_and_adam(P):
    """An instance without points gets a zero loss and gradient, and Adam leaves its s
    where it is (its locality term is zero at the anchor); the others match the oracle."""
    net, bt, rows, Xis = case(3, 64, (1, 49, 30, 25, 1), 5, [40, 0, 25], [6, 0, 3], [4, 0, 2],
                              (2.0, 1.0, 1.0))
    fnet = lrnr64.make_fast(net, rows, Xis)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db, loss="mse")
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast", loss="mse")
    assert lo[1].item() == 0.0 and torch.all(ds[1] == 0) and torch.all(dbb[1] == 0)
    for i in (0, 2):
        assert abs(lo[i].item() - ro[i]) <= TOL_FP32 * abs(ro[i]), i
        assert rel(ds[i].cpu(), rs[i]) < TOL_FP32, i
    s = torch.tensor(bt.s, dtype=torch.float32, device="cuda")
    s1 = s[1].clone()
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, n_steps=3, lr=1e-2, lambda_loc=1e-3,
                    s_anchor=s.clone(), loss="l1")
    assert step.item() == 3
    assert torch.equal(s[1], s1)
    assert P.lrnr_last_device_status(model) == 0
