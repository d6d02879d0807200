"""torch.autograd wrapper of the adjoint kernel, and the captured SPInProp graph."""
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


@pytest.mark.parametrize("form", ["fast", "full"])
def test_autograd_gradient_matches_oracle(P, form):
    from paper_2410_04001_gb300.autograd import lrnr_loss
    g = synth.rng(4)
    net = synth.make_net(g, L=3, M=48, r=8)
    bt = as_f32_batch(synth.make_instances(g, net, 3, 200, 500))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    s = db.s.clone().requires_grad_(True)
    lo = lrnr_loss(s, model, db, form=form)
    w = torch.tensor([1.0, -2.0, 0.5], device="cuda")
    (lo * w).sum().backward()
    ref = lrnr64.make_fast(net, rows, Xis) if form == "fast" else net
    ro, rs, _ = lrnr64.residual_grad(ref, bt, form)
    assert rel(lo.detach().cpu(), ro) < TOL_FP32
    assert rel(s.grad.cpu(), rs * np.array([1.0, -2.0, 0.5])[:, None]) < TOL_FP32


def test_captured_spinprop_graph_equals_eager_steps(P):
    from paper_2410_04001_gb300.graph import SpinpropGraph
    g = synth.rng(6)
    net = synth.make_net(g, L=3, M=32, r=8)
    bt = as_f32_batch(synth.make_instances(g, net, 4, 100, 300))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)

    def state():
        s = db.s.clone()
        return s, torch.zeros_like(s), torch.zeros_like(s), torch.zeros(1, dtype=torch.int64, device="cuda")
    s1, m1, v1, k1 = state()
    for _ in range(6):
        P.spinprop_step(model, "fast", "fp32", db, s1, m1, v1, k1, 2, lr=1e-2)
    s2, m2, v2, k2 = state()
    gr = SpinpropGraph(model, db, s2, m2, v2, k2, n_steps=2, lr=1e-2)   # runs 2 steps eagerly
    for _ in range(5):
        gr.replay()
    torch.cuda.synchronize()
    assert k1.item() == 12 and k2.item() == 12
    assert torch.equal(s1, s2) and torch.equal(m1, m2) and torch.equal(v1, v2)


def test_captured_step_with_host_transfers(P):
    """SpinpropGraph with copy_in / copy_out: each replay takes s from pinned host
    memory, runs the step and returns s and the loss to pinned host memory.  Feeding
    every replay the s that the previous one returned reproduces the eager steps bit
    for bit, and the host copies hold the device results."""
    from paper_2410_04001_gb300.graph import SpinpropGraph
    g = synth.rng(7)
    net = synth.make_net(g, L=3, M=32, r=8)
    bt = as_f32_batch(synth.make_instances(g, net, 3, 200, 400))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    dev = torch.device("cuda")

    def state():
        s = db.s.clone()
        return s, torch.zeros_like(s), torch.zeros_like(s), torch.zeros(1, dtype=torch.int64, device=dev)
    s1, m1, v1, k1 = state()
    lo1 = torch.zeros(db.n_inst, dtype=torch.float32, device=dev)
    for _ in range(4):
        P.spinprop_step(model, "fast", "fp32", db, s1, m1, v1, k1, 1, lr=1e-2, loss_out=lo1)
    s2, m2, v2, k2 = state()
    lo2 = torch.zeros_like(lo1)
    h_in = db.s.detach().cpu().pin_memory()
    h_s, h_lo = torch.zeros_like(h_in).pin_memory(), torch.zeros(db.n_inst).pin_memory()
    gr = SpinpropGraph(model, db.with_s(s2), s2, m2, v2, k2, 1, loss_out=lo2,
                       copy_in=[(s2, h_in)], copy_out=[(h_s, s2), (h_lo, lo2)], lr=1e-2)
    torch.cuda.synchronize()                 # the warm-up ran the first step
    for _ in range(3):
        h_in.copy_(h_s)                      # the host hands the returned s back in
        gr.replay()
        torch.cuda.synchronize()
    assert k1.item() == 4 and k2.item() == 4
    assert torch.equal(s1.cpu(), h_s) and torch.equal(lo1.cpu(), h_lo)
    assert torch.equal(s1, s2) and torch.equal(m1, m2) and torch.equal(v1, v2)


@pytest.mark.parametrize("form", ["fast", "full"])
def test_autograd_gradient_matches_central_differences_of_the_kernel_loss(P, form):
    """The gradient behind lrnr_loss against central differences of lrnr_loss itself
    (FP32 forward), along a random unit direction of s per instance: (L(s + h d) -
    L(s - h d)) / 2h = <dL/ds, d> + O(h^2) + O(eps L / h).  With h = 5e-3 the truncation
    term is about 1e-5 of the derivative and the rounding term, the loss's own FP32
    error (a few 1e-7 of L, the parity tests) over h, about 1e-4 of L: held to
    1e-3 |<dL/ds, d>| + 2e-4 L."""
    from paper_2410_04001_gb300.autograd import lrnr_loss
    g = synth.rng(8)
    net = synth.make_net(g, L=3, M=48, r=8)
    bt = as_f32_batch(synth.make_instances(g, net, 3, 300, 700))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    s = db.s.clone().requires_grad_(True)
    lo = lrnr_loss(s, model, db, form=form)
    lo.sum().backward()
    d = torch.tensor(g.standard_normal(tuple(s.shape)), dtype=torch.float32, device="cuda")
    d = d / d.norm(dim=1, keepdim=True)
    h = 5e-3
    with torch.no_grad():
        lp = lrnr_loss((s + h * d).contiguous(), model, db, form=form).double()
        lm = lrnr_loss((s - h * d).contiguous(), model, db, form=form).double()
    fd = (lp - lm) / (2.0 * h)
    an = (s.grad.double() * d.double()).sum(dim=1)
    tol = 1e-3 * an.abs() + 2e-4 * lo.detach().double().abs()
    assert torch.all((fd - an).abs() <= tol), (fd, an, lo)
