"""GPU parity: the CUDA library through its C ABI against the FP64 oracle, element by
element on the same seeded inputs (FP32 path: normwise relative error <= 1e-5 per
quantity; EIM rows and bases bit-exact)."""
import numpy as np
import pytest
import torch

import synth
from oracle import adam64, eim64, lrnr64
from tests.gpu_common import (TOL_FP32, as_f32_batch, bc_err, eim_for, install_fast,
                              per_instance_rel, rel)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def make(P, net, bt):
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    return model, P.DeviceBatch.from_host(bt)


def ragged_case(L=3, M=48, r=8, seed=5):
    g = synth.rng(seed)
    net = synth.make_net(g, L=L, M=M, r=r)
    n_int = [300, 0, 129, 1, 517, 128, 64]
    n_ic = [40, 17, 0, 3, 129, 1, 0]
    n_bc = [9, 64, 65, 0, 1, 2, 0]
    beta = [5.0, 1.0, 19.0, 3.3, 7.5, 0.0, 2.0]
    nu = [0.0, 1.5, 4.9, 0.0, 2.0, 0.3, 1.0]
    rho = [0.0, 2.0, 0.1, 4.0, 0.0, 5.0, 1.0]
    bt = synth.make_batch(g, net, n_int, n_ic, n_bc, beta, nu, rho)
    return net, as_f32_batch(bt)


# --------------------------------------------------------------------- full FP32

@pytest.mark.parametrize("mu", [(5.0, 0.0, 0.0), (5.0, 1.0, 2.0)])
def test_full_fp32_residual_matches_oracle(P, mu):
    net, bt = synth.workload_convection_small()
    bt.beta[:], bt.nu[:], bt.rho[:] = mu
    bt = as_f32_batch(bt)
    model, db = make(P, net, bt)
    out = P.lrnr_residual(model, "full", "fp32", db)
    jets, R, Bic, Bbc = lrnr64.residual_eval(net, bt, "full")
    for c, k in enumerate(("u", "u_t", "u_x", "u_xx")):
        assert rel(out[k].cpu(), jets[:, c]) < TOL_FP32, k
    assert rel(out["res"].cpu(), R) < TOL_FP32
    assert rel(out["res_ic"].cpu(), Bic) < TOL_FP32
    assert bc_err(out["res_bc"].cpu(), Bbc, net, bt, "full") < TOL_FP32


@pytest.mark.parametrize("loss,w", [("mse", None), ("l1", None), ("mse", (0.5, 2.0, 3.0))])
def test_full_fp32_gradient_matches_oracle(P, loss, w):
    net, bt = synth.workload_convection_small()
    bt.nu[:], bt.rho[:] = 1.0, 2.0
    bt = as_f32_batch(bt)
    model, db = make(P, net, bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "fp32", db, loss=loss, w=w)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full", loss, w or (1.0, 1.0, 1.0))
    assert rel(lo.cpu(), ro) < TOL_FP32
    assert rel(ds.cpu(), rs) < TOL_FP32
    assert rel(dbb.cpu(), rb) < TOL_FP32


def test_full_fp32_ragged_instances(P):
    net, bt = ragged_case()
    model, db = make(P, net, bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "full", "fp32", db)
    ro, rs, rb = lrnr64.residual_grad(net, bt, "full")
    for i in range(bt.n_inst):
        assert abs(lo[i].item() - ro[i]) <= TOL_FP32 * max(abs(ro[i]), 1e-30), i
        assert rel(ds[i].cpu(), rs[i]) < TOL_FP32, i
        assert rel(dbb[i].cpu(), rb[i]) < TOL_FP32, i
    out = P.lrnr_residual(model, "full", "fp32", db)
    jets, R, Bic, Bbc = lrnr64.residual_eval(net, bt, "full")
    assert rel(out["u_xx"].cpu(), jets[:, 3]) < TOL_FP32
    assert rel(out["res"].cpu(), R) < TOL_FP32
    assert rel(out["res_ic"].cpu(), Bic) < TOL_FP32
    assert bc_err(out["res_bc"].cpu(), Bbc, net, bt, "full") < TOL_FP32


def test_gradient_is_deterministic(P):
    net, bt = ragged_case(seed=8)
    model, db = make(P, net, bt)
    a = [t.clone() for t in P.lrnr_residual_grad(model, "full", "fp32", db)]
    b = P.lrnr_residual_grad(model, "full", "fp32", db)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


# --------------------------------------------------------------------- EIM

def test_snapshots_match_oracle(P):
    g = synth.rng(3)
    net = synth.make_net(g, L=3, M=40, r=8)
    xs, ts = synth.snapshot_design(g, 2)
    s = synth.make_s(g, 2, net.sum_r)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    for l in range(net.L):
        out = P.lrnr_snapshots(model, l, torch.tensor(xs, device="cuda"), torch.tensor(ts, device="cuda"),
                               torch.tensor(s, device="cuda")).cpu().numpy()
        ref = np.concatenate([lrnr64.hidden_states(net, s[j], xs, ts, l).T for j in range(2)])
        assert np.max(np.abs(out - ref)) < 1e-13


@pytest.mark.parametrize("M,K,rh,tol", [(64, 300, 16, 0.0), (256, 1000, 16, 0.0), (37, 5, 16, 1e-12),
                                        (1024, 96, 32, 0.0)])
def test_eim_rows_and_basis_bit_exact(P, M, K, rh, tol):
    g = synth.rng(M + K)
    S = np.tanh(g.normal(size=(M, 3)) @ g.normal(size=(3, K)) + 0.3 * g.normal(size=(M, K)))
    if K < rh:
        S = g.normal(size=(M, 2)) @ g.normal(size=(2, K))   # rank 2: early stop
    ro, Xo, uo = eim64.eim_greedy(S, rh, tol)
    net = synth.make_net(g, L=1, M=M, r=4)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    rows, Xi, used = P.fastlrnr_select_rows(model, 0, torch.tensor(S.T.copy(), device="cuda"), rh, tol)
    assert used == uo
    assert np.array_equal(rows.cpu().numpy(), ro)
    assert np.array_equal(Xi.cpu().numpy().T, Xo)       # bit for bit


def test_eim_on_device_snapshots_gives_a_valid_selection(P):
    net, bt = synth.workload_convection_small()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    g = synth.rng(9)
    xs, ts = synth.snapshot_design(g, 8)
    for l in range(net.L):
        S = P.lrnr_snapshots(model, l, torch.tensor(xs, device="cuda"), torch.tensor(ts, device="cuda"),
                             torch.tensor(bt.s[:1], device="cuda"))
        rows, Xi, used = P.fastlrnr_select_rows(model, l, S, 16)
        assert used == 16 and len(set(rows.cpu().tolist())) == 16
        T = Xi.cpu().numpy()[:, rows.cpu().numpy()].T      # P^T Xi
        assert np.array_equal(np.diag(T), np.ones(16))
        assert np.array_equal(np.triu(T, 1), np.zeros((16, 16)))


# --------------------------------------------------------------------- FastLRNR

@pytest.mark.parametrize("rh", [16, 11])
def test_fast_fp32_matches_oracle(P, rh):
    net, bt = synth.workload_convection_small()
    bt.nu[:], bt.rho[:] = 1.0, 2.0
    bt = as_f32_batch(bt)
    rows, Xis, _ = eim_for(net, bt.s[0], rh)
    fnet = lrnr64.make_fast(net, rows, Xis)
    model, db = make(P, net, bt)
    install_fast(P, model, rows, Xis)
    out = P.lrnr_residual(model, "fast", "fp32", db)
    jets, R, Bic, Bbc = lrnr64.residual_eval(fnet, bt, "fast")
    for c, k in enumerate(("u", "u_t", "u_x", "u_xx")):
        assert rel(out[k].cpu(), jets[:, c]) < TOL_FP32, k
    assert rel(out["res"].cpu(), R) < TOL_FP32
    assert bc_err(out["res_bc"].cpu(), Bbc, fnet, bt, "fast") < TOL_FP32
    for loss in ("mse", "l1"):
        lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db, loss=loss)
        ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast", loss)
        assert rel(lo.cpu(), ro) < TOL_FP32
        assert rel(ds.cpu(), rs) < TOL_FP32
        assert rel(dbb.cpu(), rb) < TOL_FP32
        assert np.all(dbb.cpu().numpy()[rb == 0.0] == 0.0)


def test_fast_fp32_ragged_instances(P):
    net, bt = ragged_case(L=4, M=64, r=16, seed=12)
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    fnet = lrnr64.make_fast(net, rows, Xis)
    model, db = make(P, net, bt)
    install_fast(P, model, rows, Xis)
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db)
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast")
    for i in range(bt.n_inst):
        assert abs(lo[i].item() - ro[i]) <= TOL_FP32 * max(abs(ro[i]), 1e-30), i
        assert rel(ds[i].cpu(), rs[i]) < TOL_FP32, i
        assert rel(dbb[i].cpu(), rb[i]) < TOL_FP32, i


def test_fast_many_ragged_instances_with_empty_ones(P):
    """About 110 tiles of 27 instances, several without points (first, middle, last),
    so that the per-tile partial rows of neighbouring instances interleave in the
    reduction and some instances have no tile at all.  Loss and gradient per
    instance against the oracle on two calls in a row, then two Adam steps."""
    g = synth.rng(41)
    net = synth.make_net(g, L=3, M=48, r=16)
    n = 27
    n_int = g.integers(0, 700, size=n)
    n_ic = g.integers(0, 60, size=n)
    n_bc = g.integers(0, 40, size=n)
    for i in (0, 9, 10, 26):
        n_int[i] = n_ic[i] = n_bc[i] = 0
    bt = as_f32_batch(synth.make_batch(g, net, n_int, n_ic, n_bc, g.uniform(1, 20, n),
                                       g.uniform(0, 5, n), g.uniform(0, 5, n)))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    fnet = lrnr64.make_fast(net, rows, Xis)
    model, db = make(P, net, bt)
    install_fast(P, model, rows, Xis)
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast")
    for rep in range(2):   # tickets must be back at zero for the second call
        lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db)
        for i in range(n):
            if n_int[i] + n_ic[i] + n_bc[i] == 0:
                assert lo[i].item() == 0.0 and torch.all(ds[i] == 0) and torch.all(dbb[i] == 0)
                continue
            assert abs(lo[i].item() - ro[i]) <= TOL_FP32 * abs(ro[i]), (rep, i)
            assert rel(ds[i].cpu(), rs[i]) < TOL_FP32, (rep, i)
            assert rel(dbb[i].cpu(), rb[i]) < TOL_FP32, (rep, i)
    s = torch.tensor(bt.s, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(s)
    v = torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo = torch.zeros(n, dtype=torch.float32, device="cuda")
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, n_steps=2, lr=1e-2, loss_out=lo)
    assert step.item() == 2
    for i in range(n):
        inst = bt.instance(i)

        def lg(sv, inst=inst):
            d = dict(inst)
            d["s"] = sv
            l_, g_, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet, d)
            return l_, g_
        sr, _, _, _ = adam64.spinprop_loop(lg, inst["s"], 2, lr=1e-2)
        disp = max(np.abs(sr - inst["s"]).max(), 1e-30)
        assert np.max(np.abs(s[i].cpu().numpy() - sr)) <= 1e-3 * disp + 1e-6, i


def test_fast_equals_full_when_every_row_is_kept(P):
    g = synth.rng(31)
    net = synth.make_net(g, L=3, M=16, r=8)
    bt = as_f32_batch(synth.make_batch(g, net, 200, 33, 17, 4.0, 0.5, 1.5))
    model, db = make(P, net, bt)
    I = np.eye(16)
    install_fast(P, model, [np.arange(16)] * 3, [I] * 3)
    a = P.lrnr_residual_grad(model, "fast", "fp32", db)
    b = P.lrnr_residual_grad(model, "full", "fp32", db)
    for x, y in zip(a, b):
        assert rel(x.cpu(), y.cpu()) < 1e-6


def test_fast_requires_selected_layers(P):
    net, bt = synth.workload_convection_small(scale=0.1)
    model, db = make(P, net, bt)
    with pytest.raises(P.LrnrError) as e:
        P.lrnr_residual_grad(model, "fast", "fp32", db)
    assert e.value.status == P.binding.ENOTREADY


# --------------------------------------------------------------------- SPInProp

@pytest.mark.parametrize("form", ["fast", "full"])
def test_spinprop_steps_match_oracle_adam(P, form):
    net, bt = ragged_case(L=3, M=32, r=8, seed=21)
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    fnet = lrnr64.make_fast(net, rows, Xis)
    model, db = make(P, net, bt)
    install_fast(P, model, rows, Xis)
    s = torch.tensor(bt.s, dtype=torch.float32, device="cuda")
    anchor = s.clone()
    m = torch.zeros_like(s)
    v = torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo = torch.zeros(bt.n_inst, dtype=torch.float32, device="cuda")
    n, lr, lam = 5, 1e-2, 1e-3
    P.spinprop_step(model, form, "fp32", db, s, m, v, step, n_steps=n, lr=lr, lambda_loc=lam,
                    s_anchor=anchor, loss_out=lo)
    assert step.item() == n
    ref = fnet if form == "fast" else net
    for i in range(bt.n_inst):
        inst = bt.instance(i)
        fwd = (lrnr64.fast_forward, lrnr64.fast_backward) if form == "fast" else (lrnr64.full_forward, lrnr64.full_backward)

        def lg(sv, inst=inst, fwd=fwd):
            d = dict(inst)
            d["s"] = sv
            l_, g_, _ = lrnr64.instance_loss_grad(fwd[0], fwd[1], ref, d)
            return l_, g_
        sr, _, _, lr_ = adam64.spinprop_loop(lg, inst["s"], n, lr=lr, lam=lam, anchor=inst["s"])
        # Adam moves each coordinate by about lr per step: compare the displacement
        disp = np.abs(sr - inst["s"]).max()
        assert np.max(np.abs(s[i].cpu().numpy() - sr)) <= 1e-3 * disp + 1e-6, i
        assert abs(lo[i].item() - lr_) <= 1e-4 * abs(lr_) + 1e-7, i


def test_spinprop_beyond_one_grid_round_matches_oracle_adam(P):
    """Two instances with more tiles than one round of the FastLRNR grid (so the
    reduction and Adam run as the separate cluster kernel, not inside the tile
    kernel), with the locality term: s after 4 steps and the last loss against the
    oracle's Adam loop."""
    g = synth.rng(23)
    net = synth.make_net(g, L=3, M=32, r=8)
    bt = as_f32_batch(synth.make_batch(g, net, [31000, 11000], [700, 300], [300, 129],
                                       [5.0, 2.0], [1.0, 0.5], [2.0, 0.0]))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    fnet = lrnr64.make_fast(net, rows, Xis)
    model, db = make(P, net, bt)
    install_fast(P, model, rows, Xis)
    assert db.n_points > 2 * 152 * 128
    s = torch.tensor(bt.s, dtype=torch.float32, device="cuda")
    anchor = s.clone()
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo = torch.zeros(bt.n_inst, dtype=torch.float32, device="cuda")
    n, lr, lam = 4, 1e-2, 1e-3
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, n_steps=n, lr=lr, lambda_loc=lam,
                    s_anchor=anchor, loss_out=lo)
    assert step.item() == n
    for i in range(bt.n_inst):
        inst = bt.instance(i)

        def lg(sv, inst=inst):
            d = dict(inst)
            d["s"] = sv
            l_, g_, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet, d)
            return l_, g_
        sr, _, _, lr_ = adam64.spinprop_loop(lg, inst["s"], n, lr=lr, lam=lam, anchor=inst["s"])
        disp = np.abs(sr - inst["s"]).max()
        assert np.max(np.abs(s[i].cpu().numpy() - sr)) <= 1e-3 * disp + 1e-6, i
        assert abs(lo[i].item() - lr_) <= 1e-4 * abs(lr_) + 1e-7, i
    assert P.lrnr_last_device_status(model) == 0


# --------------------------------------------------------------------- full-size

def test_cdr_single_full_size_fast_and_full(P):
    """The 65,536 + 2,048 + 1,024-pair CDR workload at full size, both forms, every
    precision (FP32 1e-5, split-BF16 1e-5, TF32 2.5e-3, BF16 2e-2), in the launch
    configuration the benchmark times; and the benchmark's SPInProp step (one Adam
    step through the reduced network) against the oracle's Adam step."""
    net, bt = synth.workload_cdr_single()
    bt = as_f32_batch(bt)
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    fnet = lrnr64.make_fast(net, rows, Xis)
    model, db = make(P, net, bt)
    install_fast(P, model, rows, Xis)
    tol = {"fp32": TOL_FP32, "bf16x3": 1e-5, "tf32": 2.5e-3, "bf16": 2e-2}
    oracle = {}
    for form, ref in (("fast", fnet), ("full", net)):
        ro, rs, rb = oracle[form] = lrnr64.residual_grad(ref, bt, form)
        for prec in ("fp32", "bf16x3", "tf32", "bf16"):
            lo, ds, dbb = P.lrnr_residual_grad(model, form, prec, db)
            assert rel(lo.cpu(), ro) < tol[prec], (form, prec)
            assert rel(ds.cpu(), rs) < tol[prec], (form, prec, rel(ds.cpu(), rs))
            assert rel(dbb.cpu(), rb) < tol[prec], (form, prec, rel(dbb.cpu(), rb))
    # one Adam step (bias-corrected, step 1): coordinate k moves by lr g_k / (|g_k| + eps);
    # the smallest |g_k| here is 4e-6 of ||g|| (1.7e-7), where the FP32 gradient error
    # (about 3e-7 ||g||) changes the move by up to 4e-3 lr: tolerance 1e-2 lr
    s = torch.tensor(bt.s, dtype=torch.float32, device="cuda")
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo = torch.zeros(1, dtype=torch.float32, device="cuda")
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, 1, lr=1e-3, loss_out=lo)
    sr, _, _ = adam64.adam_step(bt.s[0], np.zeros_like(bt.s[0]), np.zeros_like(bt.s[0]), 1,
                                oracle["fast"][1][0], lr=1e-3)
    disp = np.abs(sr - bt.s[0]).max()
    assert np.max(np.abs(s[0].cpu().numpy() - sr)) <= 1e-2 * disp
    assert abs(lo.item() - oracle["fast"][0][0]) <= 1e-5 * abs(oracle["fast"][0][0])
    assert P.lrnr_last_device_status(model) == 0
