"""GPU parity of the tcgen05 full-width path (BF16, TF32 and split-BF16 operands,
FP32 accumulation) against the FP64 oracle.  Tolerances (normwise relative error per
quantity): BF16 2e-2, TF32 2.5e-3 (its unit roundoff 2^-11 is 8 times smaller than
BF16's 2^-8), split-BF16 1e-5."""
import numpy as np
import pytest

import synth
from oracle import lrnr64
from tests.gpu_common import as_f32_batch, bc_err, rel

pytestmark = pytest.mark.gpu

TOL = {"bf16": 2e-2, "tf32": 2.5e-3, "bf16x3": 1e-5}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def cdr_case(L=3, M=96, r=16, n=(700, 70, 40), seed=41, mu=(5.0, 1.0, 2.0)):
    g = synth.rng(seed)
    net = synth.make_net(g, L=L, M=M, r=r)
    bt = synth.make_batch(g, net, *n, *mu)
    return net, as_f32_batch(bt)


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
def test_tc_residual_matches_oracle(P, prec):
    net, bt = cdr_case()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    out = P.lrnr_residual(model, "full", prec, db)
    jets, R, Bic, Bbc = lrnr64.residual_eval(net, bt, "full")
    for c, k in enumerate(("u", "u_t", "u_x", "u_xx")):
        assert rel(out[k].cpu(), jets[:, c]) < TOL[prec], (k, rel(out[k].cpu(), jets[:, c]))
    assert rel(out["res"].cpu(), R) < TOL[prec]
    assert rel(out["res_ic"].cpu(), Bic) < TOL[prec]
    assert bc_err(out["res_bc"].cpu(), Bbc, net, bt, "full") < TOL[prec]
    assert P.lrnr_last_device_status(model) == 0


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
@pytest.mark.parametrize("shape", [(3, 96, 16), (2, 64, 32), (4, 100, 8)])
def test_tc_gradient_matches_oracle(P, prec, shape):
    L, M, r = shape
    net, bt = cdr_case(L=L, M=M, r=r, seed=L * M + r)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", prec, db)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full")
    assert rel(lo.cpu(), ro) < TOL[prec]
    assert rel(ds.cpu(), rs) < TOL[prec], rel(ds.cpu(), rs)
    assert rel(dbb.cpu(), rb) < TOL[prec], rel(dbb.cpu(), rb)
    assert P.lrnr_last_device_status(model) == 0


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
@pytest.mark.parametrize("shape", [(2, 32, 16), (3, 20, 8), (1, 32, 16), (2, 16, 16)])
def test_tc_single_chunk_layers(P, prec, shape):
    """Widths of one chunk (32 columns in BF16 / TF32, 16 in split-BF16; M = 20 a ragged
    one) and a single hidden layer: the chunk loops without a next chunk to issue or
    prefetch.  Loss, dL/ds and dL/db against the oracle."""
    L, M, r = shape
    net, bt = cdr_case(L=L, M=M, r=r, n=(300, 40, 20), seed=100 + L * M + r)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", prec, db)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full")
    assert rel(lo.cpu(), ro) < TOL[prec]
    assert rel(ds.cpu(), rs) < TOL[prec], rel(ds.cpu(), rs)
    assert rel(dbb.cpu(), rb) < TOL[prec], rel(dbb.cpu(), rb)
    assert P.lrnr_last_device_status(model) == 0


def test_tc_ragged_instances(P):
    g = synth.rng(17)
    net = synth.make_net(g, L=3, M=64, r=16)
    bt = as_f32_batch(synth.make_batch(g, net, [300, 0, 129, 1, 517], [40, 17, 0, 3, 129],
                                       [9, 64, 65, 0, 1], [5.0, 1.0, 19.0, 3.3, 7.5],
                                       [0.0, 1.5, 4.9, 0.0, 2.0], [0.0, 2.0, 0.1, 4.0, 0.0]))
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "bf16x3", db)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full")
    for i in range(bt.n_inst):
        assert rel(ds[i].cpu(), rs[i]) < 1e-5, i
        assert rel(dbb[i].cpu(), rb[i]) < 1e-5, i
        assert abs(lo[i].item() - ro[i]) <= 1e-5 * abs(ro[i]), i


# ----------------------------------------------------------------- FastLRNR on tcgen05

@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
@pytest.mark.parametrize("shape", [(3, 96, 16, 16), (4, 64, 8, 11), (2, 80, 32, 16)])
def test_fast_tc_gradient_matches_oracle(P, prec, shape):
    """The reduced network (width r-hat, Eq. 2.8) on the tensor cores, 16-column
    chunks: loss, dL/ds and dL/db (scattered to the EIM rows) against the oracle's
    FastLRNR; r-hat = 11 leaves zero padding rows; rank 32 into 16 rows runs
    split-BF16 with its three-piece activations in tensor memory."""
    from tests.gpu_common import eim_for, install_fast
    L, M, r, rh = shape
    tol = TOL[prec]
    net, bt = cdr_case(L=L, M=M, r=r, seed=7 * L + M + rh)
    rows, Xis, _ = eim_for(net, bt.s[0], rh)
    fnet = lrnr64.make_fast(net, rows, Xis)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", prec, db)
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast")
    assert rel(lo.cpu(), ro) < tol
    assert rel(ds.cpu(), rs) < tol, rel(ds.cpu(), rs)
    assert rel(dbb.cpu(), rb) < tol, rel(dbb.cpu(), rb)
    assert np.all(dbb.cpu().numpy()[rb == 0.0] == 0.0)   # rows outside P get nothing
    out = P.lrnr_residual(model, "fast", prec, db)
    jets, R, _, _ = lrnr64.residual_eval(fnet, bt, "fast")
    assert rel(out["u"].cpu(), jets[:, 0]) < tol
    assert rel(out["res"].cpu(), R) < tol
    assert P.lrnr_last_device_status(model) == 0


def test_fast_tc_spinprop_matches_fp32_kernel(P):
    """Adam steps through the reduced network in split-BF16 on the tensor cores and
    in FP32 on the CUDA cores agree (both within 1e-5 of the FP64 gradient)."""
    from tests.gpu_common import eim_for, install_fast
    import torch
    net, bt = cdr_case(L=3, M=64, r=16, seed=5)
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    out = {}
    for prec in ("fp32", "bf16x3"):
        s = db.s.clone()
        m, v = torch.zeros_like(s), torch.zeros_like(s)
        k = torch.zeros(1, dtype=torch.int64, device="cuda")
        P.spinprop_step(model, "fast", prec, db, s, m, v, k, n_steps=5, lr=1e-2)
        assert k.item() == 5
        out[prec] = s.cpu().numpy()
    disp = np.abs(out["fp32"] - bt.s).max()
    assert np.max(np.abs(out["bf16x3"] - out["fp32"])) <= 1e-3 * disp + 1e-6
