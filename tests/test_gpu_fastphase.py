"""The fast phase as the paper runs it (Sec. 3.2 Eq. 3.6-3.7, Sec. 4) on the paper's
convection architecture in shape: width M = 4,000, ranks r = (1, 5, 5, 3, 1), EIM with
rhat = 5 rows per layer from exact-LRNR snapshots at the 4 x 3 sample grid and its
perturbations for several coefficient draws, then Adam steps of the l1 fast loss
plus the l1 locality term through the reduced network (SPInProp), then the
solution on the full-width network with the trained coefficients.

Against the FP64 oracle: the device snapshots against the oracle's exact-LRNR
states, the device EIM rows against the oracle's greedy on the oracle's snapshots;
every Adam step from the same state; the full-width solution at the trained
coefficients."""
import numpy as np
import pytest
import torch

import synth
from oracle import adam64, eim64, lrnr64
from tests.gpu_common import TOL_FP32, as_f32_batch, as_f32_net, install_fast, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def test_fast_phase_on_the_paper_convection_shape(P):
    from paper_2410_04001_gb300 import fastphase
    net, bx, bt = synth.workload_paper_d1(M=4000, n_tune=2048)
    net = as_f32_net(net)
    bx, bt = as_f32_batch(bx), as_f32_batch(bt)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    # snapshots: the 12 sample points and 8 perturbations of each, for 4 draws of s
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    s0 = bx.s[0]
    draws = np.stack([s0] + [s0 * (1.0 + 0.1 * g.standard_normal(s0.shape)) for _ in range(3)])
    dev = torch.device("cuda")
    xs_d, ts_d = torch.tensor(xs, device=dev), torch.tensor(ts, device=dev)
    sd_d = torch.tensor(draws, device=dev)
    got = fastphase.build_reduced(model, xs_d, ts_d, sd_d, rhat=5)
    rows, Xis = [], []
    for l in range(net.L):
        S = P.lrnr_snapshots(model, l, xs_d, ts_d, sd_d).cpu().numpy().T
        So = np.concatenate([lrnr64.hidden_states(net, d, xs, ts, l) for d in draws], axis=1)
        assert np.max(np.abs(S - So)) < 1e-12
        p, Xi, used = eim64.eim_greedy(So, 5)
        assert got[l][1] == used == 5
        assert np.array_equal(got[l][0].cpu().numpy(), p), l
        rows.append(p)
        Xis.append(Xi)
    fnet = lrnr64.make_fast(net, rows, Xis)
    # the steps below compare the same reduced network: the oracle's rows and bases
    # installed on the device (its own bases differ from them at rounding level)
    install_fast(P, model, rows, Xis)

    # Adam steps of the fast loss + locality, one at a time from the device state
    dX = P.DeviceBatch.from_host(bx)
    s = dX.s.clone()
    anchor = s.clone()
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device=dev)
    lo = torch.zeros(1, dtype=torch.float32, device=dev)
    lr, lam = 1e-2, 1e-3
    inst = bx.instance(0)
    for k in range(1, 11):
        s_prev = s[0].double().cpu().numpy()
        m_prev, v_prev = m[0].double().cpu().numpy(), v[0].double().cpu().numpy()
        P.spinprop_step(model, "fast", "fp32", dX, s, m, v, step, n_steps=1, lr=lr,
                        lambda_loc=lam, s_anchor=anchor, loss="l1", loss_out=lo)
        d = dict(inst)
        d["s"] = s_prev
        lf, gf, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet, d,
                                              loss="l1")
        lt, gl = adam64.locality_term(s_prev, inst["s"], lam)
        s_ref, _, _ = adam64.adam_step(s_prev, m_prev, v_prev, k, gf + gl, lr)
        assert np.max(np.abs(s[0].cpu().numpy() - s_ref)) <= 1e-3 * lr + 1e-6, k
        assert abs(lo.item() - (lf + lt)) <= 1e-5 * abs(lf + lt), k
    assert step.item() == 10

    # the solution on the full-width network at the trained coefficients
    de = P.DeviceBatch.from_host(bt)
    out = fastphase.fast_solution(model, de, s)
    s_fast = s[0].double().cpu().numpy()
    jets, _ = lrnr64.full_forward(net, s_fast, bt.x_int, bt.t_int)
    # Every output here is a sum of 4,000 FP32 products per layer, four layers deep,
    # that comes out about 30 times smaller than its summands (u ~ 0.03 from hidden
    # states ~ 0.5): the FP32 result is good to about 1e-6 of the summands' scale,
    # which is 2e-5 of u itself, so the bound for this width is 1e-4.
    wide = 10 * TOL_FP32
    assert rel(out["u"].cpu().numpy(), jets[:, 0]) <= wide
    assert rel(out["u_x"].cpu().numpy(), jets[:, 2]) <= wide
    assert rel(out["res"].cpu().numpy(), jets[:, 1] + 7.0 * jets[:, 2]) <= wide
