"""Point sharding within an instance on the GPU (the per-rank half of the
data-parallel step; the collective is covered on CPU ranks in test_shard_gloo.py):
every shard evaluated with the whole instances' counts (lrnr_batch.norm) gives
partial losses and gradients whose sum is the unsharded result, and the Adam update
applied to that sum (lrnr_adam_update) follows the oracle's Adam loop.  Also the
device-side check of batch offsets."""
import numpy as np
import pytest
import torch

import synth
from oracle import adam64, lrnr64
from paper_2410_04001_gb300 import shard
from tests.gpu_common import TOL_FP32, as_f32_batch, eim_for, install_fast, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def _case(P, seed=31):
    g = synth.rng(seed)
    net = synth.make_net(g, L=3, M=48, r=16)
    bt = as_f32_batch(synth.make_batch(g, net, [5000, 1, 700], [300, 9, 0], [120, 5, 33],
                                       [5.0, 2.0, 9.0], [1.0, 0.0, 2.0], [2.0, 1.0, 0.0]))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    return net, bt, model, lrnr64.make_fast(net, rows, Xis)


@pytest.mark.parametrize("form,prec", [("fast", "fp32"), ("full", "fp32"), ("full", "bf16x3")])
@pytest.mark.parametrize("world", [2, 3])
def test_point_shards_add_up_to_the_instance(P, form, prec, world):
    net, bt, model, fnet = _case(P)
    whole = P.lrnr_residual_grad(model, form, prec, P.DeviceBatch.from_host(bt))
    tot = None
    for r in range(world):
        part, counts = shard.point_shard(bt, world, r)
        out = P.lrnr_residual_grad(model, form, prec, P.DeviceBatch.from_host(part, norm=counts))
        tot = [o.double() for o in out] if tot is None else [a + o.double() for a, o in zip(tot, out)]
    ref = lrnr64.residual_grad(fnet if form == "fast" else net, bt, form)
    for a, b, c in zip(tot, whole, ref):
        assert rel(a.cpu().numpy(), b.double().cpu().numpy()) < 2e-6
        assert rel(a.cpu().numpy(), c) < TOL_FP32
    assert P.lrnr_last_device_status(model) == 0


def test_sharded_spinprop_step_follows_the_oracle_adam_loop(P):
    """Three steps of shard.sharded_spinprop_step on one rank (no collective: the
    shard is the whole batch with its own counts) against the oracle's Adam loop."""
    net, bt, model, fnet = _case(P, seed=32)
    part, counts = shard.point_shard(bt, 1, 0)
    s = torch.tensor(bt.s, dtype=torch.float32, device="cuda")
    anchor = s.clone()
    db = P.DeviceBatch.from_host(part, norm=counts).with_s(s)
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    lo = torch.zeros(bt.n_inst, dtype=torch.float32, device="cuda")
    n, lr, lam = 3, 1e-2, 1e-3
    for _ in range(n):
        shard.sharded_spinprop_step(model, "fast", "fp32", db, s, m, v, step, None, lr=lr,
                                    lambda_loc=lam, s_anchor=anchor, loss_out=lo)
    assert step.item() == n
    for i in range(bt.n_inst):
        inst = bt.instance(i)

        def lg(sv, inst=inst):
            l_, g_, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet,
                                                  dict(inst, s=sv))
            return l_, g_
        sr, _, _, lr_ = adam64.spinprop_loop(lg, inst["s"], n, lr=lr, lam=lam, anchor=inst["s"])
        disp = np.abs(sr - inst["s"]).max()
        assert np.max(np.abs(s[i].cpu().numpy() - sr)) <= 1e-3 * disp + 1e-6, i
        assert abs(lo[i].item() - lr_) <= 1e-4 * abs(lr_) + 1e-7, i
    assert P.lrnr_last_device_status(model) == 0


def test_adam_update_matches_oracle_step(P):
    g = synth.rng(33)
    n_inst, sum_r = 5, 300
    s0 = g.uniform(0.5, 1.5, (n_inst, sum_r))
    gr = g.standard_normal((n_inst, sum_r))
    m0 = 0.1 * g.standard_normal((n_inst, sum_r))
    v0 = g.uniform(0.0, 0.2, (n_inst, sum_r))
    f = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    s, m, v, gd = f(s0), f(m0), f(v0), f(gr)
    anchor = f(s0 + 1e-3 * g.standard_normal((n_inst, sum_r)))
    step = torch.full((1,), 6, dtype=torch.int64, device="cuda")
    lin = f(g.uniform(0.0, 1.0, n_inst))
    lout = torch.zeros(n_inst, dtype=torch.float32, device="cuda")
    P.lrnr_adam_update(gd, s, m, v, step, lr=1e-2, lambda_loc=0.1, s_anchor=anchor, loss_in=lin,
                       loss_out=lout)
    assert step.item() == 7
    a64 = anchor.double().cpu().numpy()
    s32 = s0.astype(np.float32).astype(np.float64)
    lt, lg = adam64.locality_term(s32, a64, 0.1)
    sr, mr, vr = adam64.adam_step(s32, m0.astype(np.float32).astype(np.float64),
                                  v0.astype(np.float32).astype(np.float64), 7,
                                  gr.astype(np.float32).astype(np.float64) + lg, lr=1e-2)
    assert np.max(np.abs(s.cpu().numpy() - sr)) < 1e-6
    assert rel(m.cpu().numpy(), mr) < 1e-6 and rel(v.cpu().numpy(), vr) < 1e-6
    assert rel(lout.cpu().numpy(), lin.double().cpu().numpy() + lt) < 1e-6


@pytest.mark.parametrize("form,prec", [("fast", "fp32"), ("full", "fp32"), ("full", "bf16")])
def test_offsets_past_the_totals_are_refused_on_the_device(P, form, prec):
    """Offsets that end past the host totals or decrease: no point is read, the
    outputs are zero and the device status says EINVAL; the next good call is exact."""
    net, bt, model, _ = _case(P, seed=34)
    db = P.DeviceBatch.from_host(bt)
    good = P.lrnr_residual_grad(model, form, prec, db)
    for bad_off in (np.array([0, 5000, 5001, 5701 + 1000]), np.array([0, 5000, 4000, 5701])):
        t = dict(db.tensors)
        t["int_off"] = torch.tensor(bad_off, dtype=torch.int64, device="cuda")
        bad = P.DeviceBatch(db.n_inst, **t)
        lo, ds, dbb = P.lrnr_residual_grad(model, form, prec, bad)
        assert P.lrnr_last_device_status(model) == P.binding.EINVAL
        assert float(lo.abs().max()) == 0.0 and float(ds.abs().max()) == 0.0
    again = P.lrnr_residual_grad(model, form, prec, db)
    for a, b in zip(again, good):
        assert torch.equal(a, b)
    assert P.lrnr_last_device_status(model) == 0
