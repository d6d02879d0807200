"""The paper's convection-diffusion-reaction network in shape (ranks r = (1, 49, 30,
25, 1), padded to 64): the tensor-core kernels in BF16 (32-column chunks, one CTA per
SM) for the full-width network and for its EIM-reduced form, against the FP64 oracle;
the reduced form also in FP32 (the reduced-coordinate kernel, rhat-dimensional jets);
the full-width FP32 kernel, which keeps a point's rank-r jets in registers, reports
ENOTSUP at this rank, and so does split-BF16 (its operands exceed shared memory)."""
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
    for form, prec in (("full", "fp32"), ("full", "bf16x3")):
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
