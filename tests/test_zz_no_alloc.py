"""The allocation-free entry point (lrnr_residual_grad_noalloc) against the ordinary
one.  Callers that cannot allocate device memory (a global-mode graph capture, a
memory budget owned by another allocator) use it; it must give the same FastLRNR
FP32 loss and gradient from its fixed scratch, on repeated calls, and refuse
batches larger than that scratch.  Kept in a file of its own, collected last."""
import numpy as np
import pytest
import torch

import synth
from tests.gpu_common import TOL_FP32, as_f32_batch, eim_for, install_fast, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def _model(P):
    g = synth.rng(303)
    net = synth.make_net(g, L=4, M=96, r=16)
    bt = as_f32_batch(synth.make_batch(g, net, [3000, 517, 0], [200, 0, 33], [64, 9, 1],
                                       [5.0, 12.0, 2.0], [1.0, 0.0, 3.0], [2.0, 1.0, 0.5]))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    return model, P.DeviceBatch.from_host(bt)


@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_noalloc_matches_allocating_entry_on_two_calls(P, loss):
    model, db = _model(P)
    ref = P.lrnr_residual_grad(model, "fast", "fp32", db, loss=loss)
    outs = [P.lrnr_residual_grad_noalloc(model, db, loss=loss) for _ in range(2)]
    torch.cuda.synchronize()
    for out in outs:
        for a, b in zip(out, ref):
            assert rel(a.cpu().numpy(), b.cpu().numpy()) <= TOL_FP32
    assert P.lrnr_last_device_status(model) == 0


def test_noalloc_refuses_batches_beyond_its_scratch(P):
    model, db = _model(P)
    big = P.DeviceBatch(db.n_inst, **db.tensors)
    big.struct.n_int = 1 << 31           # host-side total only: rejected before any GPU work
    with pytest.raises(P.LrnrError) as e:
        P.lrnr_residual_grad_noalloc(model, big)
    assert e.value.status == P.binding.ETOOBIG
