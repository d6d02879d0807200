"""The larger workloads at full size, in the launch configuration the benchmark uses,
checked on outputs the FP64 oracle can compute one by one (sampled instances or
points) and on properties that hold at any size."""
import numpy as np
import pytest
import torch

import synth
from oracle import adam64, eim64, lrnr64
from tests.gpu_common import TOL_FP32, as_f32_batch, jet_err, jet_magnitudes, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def select_on_device(P, model, net, s0, rhat=16):
    """FastLRNR construction on the device: the device snapshots match the oracle's
    exact-LRNR states; the device EIM, run on the oracle's snapshot matrix (the one
    matrix both sides take), gives the oracle's rows and bases bit for bit.  (Run on
    its own snapshots instead, it may pick other rows at the deep layers: there the
    snapshot spectra fall below rounding after about ten modes, and the late greedy
    steps choose among residuals at the rounding level.)"""
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    xs_d, ts_d = torch.tensor(xs, device="cuda"), torch.tensor(ts, device="cuda")
    rows, Xis = [], []
    for l in range(net.L):
        S = P.lrnr_snapshots(model, l, xs_d, ts_d, torch.tensor(s0[None, :], device="cuda"))
        So = lrnr64.hidden_states(net, s0, xs, ts, l)
        assert np.max(np.abs(S.cpu().numpy().T - So)) < 1e-13
        r_d, X_d, used = P.fastlrnr_select_rows(model, l, torch.tensor(So.T.copy(), device="cuda"),
                                                rhat)
        p, Xi, u = eim64.eim_greedy(So, rhat)
        assert used == u and np.array_equal(r_d.cpu().numpy(), p)
        assert np.array_equal(X_d.cpu().numpy().T, Xi)
        rows.append(p)
        Xis.append(Xi)
    return lrnr64.make_fast(net, rows, Xis)


def test_batched_512_instances_fast(P):
    """512 CDR instances, per-instance s, log-uniform counts (~7.9 M points)."""
    net, bt = synth.workload_batched()
    bt = as_f32_batch(bt)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    fnet = select_on_device(P, model, net, bt.s[0])
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db)
    lo, ds, dbb = lo.cpu().numpy(), ds.cpu().numpy(), dbb.cpu().numpy()
    assert np.all(np.isfinite(lo)) and P.lrnr_last_device_status(model) == 0
    for i in (0, 1, 137, 300, 511):
        inst = bt.instance(i)
        ro, rs, rb = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet, inst)
        assert abs(lo[i] - ro) <= TOL_FP32 * abs(ro), i
        assert rel(ds[i], rs) < TOL_FP32, i
        assert rel(dbb[i], rb) < TOL_FP32, i


# Jet tolerance per precision (normwise error over the sampled points, measured
# against each channel's rounding scale, see gpu_common.jet_magnitudes).
JET_TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "tf32": 2.5e-3, "bf16": 2e-2}


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-5), ("tf32", 2.5e-3),
                                      ("bf16", 2e-2)])
def test_adjoint_stress_full_width(P, prec, tol):
    """M = 1,024, r = 32, L = 6, 262,144 points: jets at sampled points over the whole
    batch; the gradient on a 4,096-point sub-batch against the oracle; and, over the
    whole batch, additivity of the l1 gradient over a split of the points."""
    net, bt = synth.workload_adjoint_stress()
    bt = as_f32_batch(bt)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt)
    out = P.lrnr_residual(model, "full", prec, db)
    idx = np.arange(0, bt.x_int.shape[0], 512)
    u, _ = lrnr64.full_forward(net, bt.s[0], bt.x_int[idx], bt.t_int[idx])
    # at this depth and width the derivative channels are small results of large
    # cancelling sums (u_xx ~ 1e-13): their error is measured against their magnitude
    mag = jet_magnitudes(net, bt.s[0], bt.x_int[idx], bt.t_int[idx])
    for c, k in enumerate(("u", "u_t", "u_x", "u_xx")):
        assert jet_err(out[k].cpu().numpy()[idx], u[:, c], mag[:, c]) < JET_TOL[prec], k
    # gradient on a sub-batch
    sub = synth.Batch(beta=bt.beta, nu=bt.nu, rho=bt.rho, s=bt.s, int_off=np.array([0, 4096]),
                      ic_off=np.array([0, 0]), bc_off=np.array([0, 0]), x_int=bt.x_int[:4096],
                      t_int=bt.t_int[:4096], x_ic=bt.x_ic, t_bc=bt.t_bc)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", prec, P.DeviceBatch.from_host(sub))
    ro, rs, rb = lrnr64.residual_grad(net, sub, "full")
    assert rel(lo.cpu(), ro) < tol
    assert rel(ds.cpu(), rs) < tol
    assert rel(dbb.cpu(), rb) < tol
    # full size: the l1 gradient of the batch is the sum of the gradients of its halves
    n = bt.x_int.shape[0]
    halves = []
    for a, b in ((0, n // 2), (n // 2, n)):
        hb = synth.Batch(beta=bt.beta, nu=bt.nu, rho=bt.rho, s=bt.s, int_off=np.array([0, b - a]),
                         ic_off=np.array([0, 0]), bc_off=np.array([0, 0]), x_int=bt.x_int[a:b],
                         t_int=bt.t_int[a:b], x_ic=bt.x_ic, t_bc=bt.t_bc)
        halves.append(P.lrnr_residual_grad(model, "full", prec, P.DeviceBatch.from_host(hb), loss="l1"))
    whole = P.lrnr_residual_grad(model, "full", prec, db, loss="l1")
    for k in range(3):
        assert rel(whole[k].cpu(), (halves[0][k] + halves[1][k]).cpu()) < 1e-5
    assert P.lrnr_last_device_status(model) == 0


def test_spinprop_1024_instances(P):
    """1,024 instances x 16,384 points, M = 512: three fused SPInProp steps on the
    whole batch; sampled instances against the oracle's Adam loop."""
    net, bt = synth.workload_spinprop()
    bt = as_f32_batch(bt)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    fnet = select_on_device(P, model, net, bt.s[0])
    db = P.DeviceBatch.from_host(bt)
    s = db.s.clone()
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo = torch.zeros(bt.n_inst, dtype=torch.float32, device="cuda")
    n, lr = 3, 1e-3
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, n_steps=n, lr=lr, loss_out=lo)
    s, lo = s.cpu().numpy(), lo.cpu().numpy()
    assert step.item() == n and P.lrnr_last_device_status(model) == 0
    for i in (0, 511, 1023):
        inst = bt.instance(i)

        def lg(sv, inst=inst):
            l_, g_, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet,
                                                  dict(inst, s=sv))
            return l_, g_
        sr, _, _, lr_ = adam64.spinprop_loop(lg, inst["s"], n, lr=lr)
        disp = np.abs(sr - inst["s"]).max()
        assert np.max(np.abs(s[i] - sr)) <= 1e-3 * disp + 1e-7, i
        assert abs(lo[i] - lr_) <= 1e-5 * abs(lr_), i
