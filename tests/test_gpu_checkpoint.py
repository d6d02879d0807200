"""Checkpoint / resume of a SPInProp run (s, Adam moments, step counter and the
reduced network): stopping after some steps, saving, reloading into a freshly built
model and continuing gives bit for bit what the uninterrupted run gives."""
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


@pytest.mark.parametrize("method", ["eim", "deim"])
def test_resume_from_checkpoint_is_bit_identical(P, tmp_path, method):
    from paper_2410_04001_gb300 import checkpoint
    g = synth.rng(91)
    net = synth.make_net(g, L=3, M=64, r=16)
    bt = synth.make_instances(g, net, 6, 300, 3000)
    xs, ts = synth.snapshot_design(synth.rng(77), 8)
    dev = torch.device("cuda")

    def fresh():
        return P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)

    model = fresh()
    rows, Xis = [], []
    s0 = torch.tensor(bt.s[:1], device=dev)
    for l in range(net.L):
        S = P.lrnr_snapshots(model, l, torch.tensor(xs, device=dev), torch.tensor(ts, device=dev), s0)
        if method == "eim":
            r, X, _ = P.fastlrnr_select_rows(model, l, S, 12)
        else:   # POD basis + DEIM rows: a general (not triangular) P^T Xi
            r, X, _, _ = P.fastlrnr_select_rows_deim(model, l, S, 12, tol=1e-12)
        rows.append(r)
        Xis.append(X)
    db = P.DeviceBatch.from_host(bt)
    s = db.s.clone()
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device=dev)
    kw = dict(lr=1e-2, lambda_loc=1e-3, s_anchor=db.s, loss="l1")
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, n_steps=4, **kw)
    path = tmp_path / "run.npz"
    checkpoint.save(path, s, m, v, step, rows, Xis)
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, step, n_steps=3, **kw)

    model2 = fresh()
    s2, m2, v2, step2 = checkpoint.load(path, model2)
    assert step2.item() == 4
    P.spinprop_step(model2, "fast", "fp32", db, s2, m2, v2, step2, n_steps=3, **kw)
    torch.cuda.synchronize()
    assert torch.equal(s, s2) and torch.equal(m, m2) and torch.equal(v, v2)
    assert step.item() == step2.item() == 7
