"""Edge cases and degenerate inputs through the C ABI: one hidden layer, a rank-one
input layer, the closed-form convection invariant, empty batches, non-finite
inputs and invalid EIM arguments (host-side errors; nothing faults the GPU)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import lrnr64
from tests.gpu_common import TOL_FP32, as_f32_batch, eim_for, install_fast, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


@pytest.mark.parametrize("form", ["full", "fast"])
def test_single_hidden_layer(P, form):
    g = synth.rng(71)
    net = synth.make_net(g, L=1, M=40, r=8)
    bt = as_f32_batch(synth.make_batch(g, net, 333, 21, 17, 3.0, 0.7, 1.1))
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    ref = net
    if form == "fast":
        rows, Xis, _ = eim_for(net, bt.s[0], 12)
        install_fast(P, model, rows, Xis)
        ref = lrnr64.make_fast(net, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, form, "fp32", db)
    ro, rs, rb = lrnr64.residual_grad(ref, bt, form)
    assert rel(lo.cpu(), ro) < TOL_FP32 and rel(ds.cpu(), rs) < TOL_FP32 and rel(dbb.cpu(), rb) < TOL_FP32


@pytest.mark.parametrize("form,prec", [("full", "fp32"), ("full", "bf16x3"), ("fast", "fp32")])
def test_network_of_x_minus_beta_t_has_zero_convection_residual(P, form, prec):
    """With r_1 = 1 and V^1 proportional to (1, -beta) the network is a function of
    x - beta t, so u_t + beta u_x vanishes up to rounding, whatever the other weights."""
    beta = 6.0
    g = synth.rng(72)
    net = synth.make_net(g, L=3, M=64, r=16, r1=1)
    net.V[0] = np.array([[0.9], [-0.9 * beta]])
    bt = as_f32_batch(synth.make_batch(g, net, 2000, 0, 0, beta, 0.0, 0.0))
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    if form == "fast":
        rows, Xis, _ = eim_for(net, bt.s[0], 16)
        install_fast(P, model, rows, Xis)
    out = P.lrnr_residual(model, form, prec, P.DeviceBatch.from_host(bt))
    ux = out["u_x"].cpu().numpy().astype(np.float64)
    R = out["res"].cpu().numpy()
    assert np.linalg.norm(ux) > 0
    # R = u_t + beta u_x cancels two channels computed independently: its size is the
    # channels' relative error (FP32 and split-BF16 ~1e-7)
    tol = 1e-5
    assert np.linalg.norm(R) <= tol * beta * np.linalg.norm(ux)


def test_empty_point_sets_give_zero_loss_and_gradient(P):
    g = synth.rng(73)
    net = synth.make_net(g, L=2, M=32, r=8)
    bt = as_f32_batch(synth.make_batch(g, net, [0, 50], [0, 7], [0, 3], [1.0, 2.0], [0.5, 0.5],
                                       [0.0, 1.0]))
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "fp32", P.DeviceBatch.from_host(bt))
    assert lo[0].item() == 0.0 and torch.all(ds[0] == 0) and torch.all(dbb[0] == 0)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full")
    assert rel(ds[1].cpu(), rs[1]) < TOL_FP32


def test_non_finite_input_is_reported_not_fatal(P):
    g = synth.rng(74)
    net = synth.make_net(g, L=2, M=32, r=8)
    bt = as_f32_batch(synth.make_batch(g, net, 300, 10, 5, 2.0, 0.5, 0.5))
    bt.x_int[17] = math.nan
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    P.lrnr_residual_grad(model, "full", "fp32", P.DeviceBatch.from_host(bt))
    assert P.lrnr_last_device_status(model) == P.binding.ENONFINITE
    assert P.lrnr_last_device_status(model) == 0          # read and cleared
    # the context stays usable
    bt.x_int[17] = 1.0
    lo, _, _ = P.lrnr_residual_grad(model, "full", "fp32", P.DeviceBatch.from_host(bt))
    assert torch.isfinite(lo).all()


def test_invalid_eim_arguments_are_rejected(P):
    g = synth.rng(75)
    net = synth.make_net(g, L=2, M=24, r=8)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    S = torch.tensor(g.normal(size=(40, 24)), device="cuda")
    with pytest.raises(P.LrnrError) as e:
        P.fastlrnr_select_rows(model, 0, S, rhat=33)               # more than 32 rows
    assert e.value.status == P.binding.EINVAL
    with pytest.raises(P.LrnrError) as e:
        P.fastlrnr_select_rows(model, 5, S, rhat=4)                # no such layer
    assert e.value.status == P.binding.EINVAL
    rows = torch.tensor([0, 3, 3, 7], dtype=torch.int32, device="cuda")   # repeated row
    Xi = torch.eye(24, dtype=torch.float64, device="cuda")[:4]
    with pytest.raises(P.LrnrError) as e:
        P.fastlrnr_select_rows(model, 0, rhat=4, rows_in=rows, Xi_in=Xi)
    assert e.value.status == P.binding.EINVAL
    rows = torch.tensor([0, 3, 5, 7], dtype=torch.int32, device="cuda")
    Xi = torch.zeros((4, 24), dtype=torch.float64, device="cuda")          # P^T Xi = 0
    with pytest.raises(P.LrnrError) as e:
        P.fastlrnr_select_rows(model, 0, rhat=4, rows_in=rows, Xi_in=Xi)
    assert e.value.status == P.binding.ESINGULAR


def test_unsupported_combinations_are_reported(P):
    """Rank 40 (padded to 64) runs in FP32 (four threads per point) and BF16: TF32
    and split-BF16 report LRNR_ENOTSUP."""
    g = synth.rng(76)
    net = synth.make_net(g, L=2, M=64, r=40)
    bt = synth.make_batch(g, net, 10, 2, 2, 1.0, 0.1, 0.1)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(as_f32_batch(bt))
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "fp32", db)
    ro, rs, rb = lrnr64.residual_grad(net, as_f32_batch(bt), "full")
    assert rel(ds.cpu(), rs) < 1e-5 and rel(dbb.cpu(), rb) < 1e-5 and rel(lo.cpu(), ro) < 1e-5
    for prec in ("tf32", "bf16x3"):
        with pytest.raises(P.LrnrError) as e:
            P.lrnr_residual_grad(model, "full", prec, db)
        assert e.value.status == P.binding.ENOTSUP, prec
    P.lrnr_residual_grad(model, "full", "bf16", db)


def test_peak_microbenchmarks_are_plausible(P):
    """The FP32 FMA microbenchmark reaches the unit-count peak (152 SMs x 128 lanes x 2
    flops x clock) within a few percent; the others report positive rates."""
    pk = P.lrnr_measure_peaks()
    formula = pk["sms"] * 128 * 2 * pk["sm_mhz"] * 1e6 / 1e12
    assert 0.8 * formula < max(pk["fp32_fma_tflops"], pk["fp32_fma2_tflops"]) < 1.1 * formula, (pk, formula)
    assert pk["tanh_approx_gops"] > 0 and pk["tanhf_gops"] > 0 and pk["fp64_fma_tflops"] > 0
    assert 500 < pk["sm_mhz"] < 2500


def test_wait_cap_reports_timeout_and_the_next_call_is_exact(P):
    """Failure detection without a GPU fault: a cap of zero polls on the tensor-core
    kernel's mbarrier waits makes its first wait give up; the kernel records
    LRNR_ETIMEOUT, waits for the copy and MMAs it still has outstanding and returns.
    With the cap restored the same call reproduces the earlier result bit for bit."""
    import torch
    g = synth.rng(78)
    net = synth.make_net(g, L=2, M=64, r=16)
    bt = synth.make_batch(g, net, 200, 20, 10, 5.0, 1.0, 2.0)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    ref = [t.clone() for t in P.lrnr_residual_grad(model, "full", "bf16", db)]
    assert P.lrnr_last_device_status(model) == 0
    P.lrnr_set_wait_limit(model, 0)
    P.lrnr_residual_grad(model, "full", "bf16", db)
    torch.cuda.synchronize()
    assert P.lrnr_last_device_status(model) == P.binding.ETIMEOUT
    P.lrnr_set_wait_limit(model, -1)
    again = P.lrnr_residual_grad(model, "full", "bf16", db)
    assert P.lrnr_last_device_status(model) == 0
    for a, b in zip(again, ref):
        assert torch.equal(a, b)
