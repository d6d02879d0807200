"""The paper's convection-diffusion-reaction network in shape (ranks r = (1, 49, 30,
25, 1), padded to 64): the full-width network in FP32 (the sliced kernel, four threads
per point) and in BF16 on the tensor cores (32-column chunks, one CTA per SM), the
EIM-reduced form in FP32 (the reduced-coordinate kernel, rhat-dimensional jets) and in
BF16, against the FP64 oracle; split-BF16 and TF32 report ENOTSUP at this rank (their
rank-r operands exceed shared memory)."""
import numpy as np
import pytest

import synth
from oracle import lrnr64
from tests.gpu_common import as_f32_batch, as_f32_net, eim_for, install_fast, rel

pytestmark = pytest.mark.gpu

TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def test_rank49_network_in_bf16(P):
    net, _, bt = synth.workload_paper_d2(M=192, n_tune=2048)
    net, bt = as_f32_net(net), as_f32_batch(bt)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    for form, prec in (("full", "bf16x3"), ("full", "tf32")):
        with pytest.raises(P.LrnrError) as e:
            P.lrnr_residual_grad(model, form, prec, db)
        assert e.value.status == P.binding.ENOTSUP
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "bf16", db)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full")
    err = {"loss": rel(lo.cpu(), ro), "ds": rel(ds.cpu(), rs), "db": rel(dbb.cpu(), rb)}
    assert max(err.values()) < TOL_BF16, err

    rows, Xis, _ = eim_for(net, bt.s[0], 5)
    install_fast(P, model, rows, Xis)
    fnet = lrnr64.make_fast(net, rows, Xis)
    with pytest.raises(P.LrnrError) as e:
        P.lrnr_residual_grad(model, "fast", "bf16x3", db)
    assert e.value.status == P.binding.ENOTSUP
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast")
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db)
    err = {"loss": rel(lo.cpu(), ro), "ds": rel(ds.cpu(), rs), "db": rel(dbb.cpu(), rb)}
    assert max(err.values()) < 1e-5, err
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "bf16", db)
    err = {"loss": rel(lo.cpu(), ro), "ds": rel(ds.cpu(), rs), "db": rel(dbb.cpu(), rb)}
    assert max(err.values()) < TOL_BF16, err
    assert np.all(dbb.cpu().numpy()[rb == 0.0] == 0.0)
    assert P.lrnr_last_device_status(model) == 0


@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_rank49_full_width_fp32(P, loss):
    """Full-width FP32 at padded rank 64 (four threads share a point): loss, dL/ds and
    dL/db of ragged instances with initial and periodic points (M = 100: the last
    block of 8 rows of the bias gradient is partial), and the forward outputs."""
    g = synth.rng(64)
    net = synth.make_net_ranks(g, 100, [1, 49, 30, 25, 1])
    net = as_f32_net(net)
    bt = as_f32_batch(synth.make_batch(g, net, [700, 33, 0], [50, 0, 17], [20, 7, 9],
                                       [2.0, 5.0, 1.0], [1.0, 0.0, 0.5], [1.0, 2.0, 0.0]))
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "fp32", db, loss=loss)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full", loss=loss)
    err = {"loss": rel(lo.cpu(), ro), "ds": rel(ds.cpu(), rs), "db": rel(dbb.cpu(), rb)}
    assert max(err.values()) < 1e-5, err
    out = P.lrnr_residual(model, "full", "fp32", db)
    jets, R, Bic, Bbc = lrnr64.residual_eval(net, bt, "full")
    for c, k in enumerate(("u", "u_t", "u_x", "u_xx")):
        assert rel(out[k].cpu(), jets[:, c]) < 1e-5, k
    assert rel(out["res"].cpu(), R) < 1e-5
    assert rel(out["res_ic"].cpu(), Bic) < 1e-5
    from tests.gpu_common import bc_err
    assert bc_err(out["res_bc"].cpu(), Bbc, net, bt, "full") < 1e-5
    assert P.lrnr_last_device_status(model) == 0


def test_rank32_full_width_fp32_two_threads_per_point(P):
    """Padded rank 32 (two threads per point) with a ragged batch, against the oracle."""
    g = synth.rng(32)
    net = synth.make_net(g, L=3, M=72, r=32)
    bt = as_f32_batch(synth.make_batch(g, net, [400, 129], [31, 64], [17, 1], [5.0, 2.0],
                                       [1.0, 0.3], [2.0, 1.0]))
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "fp32", db)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full")
    err = {"loss": rel(lo.cpu(), ro), "ds": rel(ds.cpu(), rs), "db": rel(dbb.cpu(), rb)}
    assert max(err.values()) < 1e-5, err
    assert P.lrnr_last_device_status(model) == 0
