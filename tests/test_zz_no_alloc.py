"""The allocation-free entry point (lrnr_residual_grad_noalloc).  Callers whose
device memory belongs to another allocator or is held to a fixed budget cannot let
the library grow a workspace with cudaMalloc; this entry point takes its scratch
from a fixed array in the library image instead.  It must give the FastLRNR FP32
loss and gradient of the ordinary entry point -- checked against the FP64 oracle
and against lrnr_residual_grad, on two calls in a row, starting from a model that
has never allocated a workspace -- follow the model's tuning, and refuse batches
larger than its scratch.  Kept in a file of its own, collected last."""
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


def _case(P):
    g = synth.rng(303)
    net = synth.make_net(g, L=4, M=96, r=16)
    bt = as_f32_batch(synth.make_batch(g, net, [3000, 517, 0], [200, 0, 33], [64, 9, 1],
                                       [5.0, 12.0, 2.0], [1.0, 0.0, 3.0], [2.0, 1.0, 0.5]))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    return model, P.DeviceBatch.from_host(bt), lrnr64.make_fast(net, rows, Xis), bt


@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_noalloc_first_on_a_fresh_model_matches_oracle_and_allocating_entry(P, loss):
    model, db, fnet, bt = _case(P)
    # the model has not run a residual / gradient pass yet: no workspace exists, so
    # these two calls can only have used the library's fixed scratch
    outs = [P.lrnr_residual_grad_noalloc(model, db, loss=loss) for _ in range(2)]
    torch.cuda.synchronize()
    ro, rs, rb = lrnr64.residual_grad(fnet, bt, "fast", loss=loss)
    for lo, ds, dbb in outs:
        assert rel(lo.cpu(), ro) <= TOL_FP32
        assert rel(ds.cpu(), rs) <= TOL_FP32
        assert rel(dbb.cpu(), rb) <= TOL_FP32
    ref = P.lrnr_residual_grad(model, "fast", "fp32", db, loss=loss)
    for out in outs:
        for a, b in zip(out, ref):
            assert rel(a.cpu().numpy(), b.cpu().numpy()) <= TOL_FP32
    assert P.lrnr_last_device_status(model) == 0


def test_noalloc_follows_the_tile_size_override(P):
    model, db, _, _ = _case(P)
    P.lrnr_set_tuning(model, "fast", "fp32", nt=64, ctas_per_sm=1)
    a = P.lrnr_residual_grad_noalloc(model, db)
    b = P.lrnr_residual_grad(model, "fast", "fp32", db)
    for x, y in zip(a, b):
        assert rel(x.cpu().numpy(), y.cpu().numpy()) <= TOL_FP32
    assert P.lrnr_last_device_status(model) == 0


def test_noalloc_refuses_batches_beyond_its_scratch(P):
    model, db, _, _ = _case(P)
    big = P.DeviceBatch(db.n_inst, **db.tensors)
    big.struct.n_int = 1 << 31           # host-side total only: rejected before any GPU work
    with pytest.raises(P.LrnrError) as e:
        P.lrnr_residual_grad_noalloc(model, big)
    assert e.value.status == P.binding.ETOOBIG
