"""The launch-shape autotuner: it installs a shape, caches it, and results change
only by rounding."""
import json

import pytest

import synth
from tests.gpu_common import TOL_FP32, as_f32_batch, eim_for, install_fast, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


@pytest.mark.parametrize("form", ["fast", "full"])
def test_autotune_installs_a_cached_shape(P, form, tmp_path):
    from paper_2410_04001_gb300.autotune import autotune
    g = synth.rng(9)
    net = synth.make_net(g, L=3, M=64, r=16)
    bt = as_f32_batch(synth.make_instances(g, net, 5, 500, 3000))
    rows, Xis, _ = eim_for(net, bt.s[0], 16)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    install_fast(P, model, rows, Xis)
    db = P.DeviceBatch.from_host(bt)
    ref = [t.clone() for t in P.lrnr_residual_grad(model, form, "fp32", db)]
    cache = tmp_path / "tune.json"
    best = autotune(model, db, form, "fp32", cache=str(cache), reps=2)
    assert best["nt"] in (32, 64, 128)
    assert best["key"] in json.loads(cache.read_text())
    got = P.lrnr_residual_grad(model, form, "fp32", db)
    for a, b in zip(got, ref):
        assert rel(a.cpu(), b.cpu()) < TOL_FP32
    again = autotune(model, db, form, "fp32", cache=str(cache))      # from the cache
    assert again["nt"] == best["nt"] and again["ctas_per_sm"] == best["ctas_per_sm"]
