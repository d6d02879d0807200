"""GPU parity of the DEIM variant (Sec. 2.2 Eq. 2.7): the POD basis of ``lrnr_pod``
(FP64 subspace iteration) against the oracle's thin SVD, the DEIM rows of
``lrnr_deim_rows`` against the oracle's DEIM (bit-exact integers), and the FastLRNR
built from them against the oracle's FastLRNR.  Snapshot matrices are made by the
oracle (or planted) and handed to both sides."""
import numpy as np
import pytest

import synth
from oracle import deim64 as D
from oracle import lrnr64
from tests.gpu_common import as_f32_batch, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def planted(seed, M, K, sig):
    g = synth.rng(seed)
    sig = np.asarray(sig, np.float64)
    Q, _ = np.linalg.qr(g.standard_normal((M, len(sig))))
    W, _ = np.linalg.qr(g.standard_normal((K, len(sig))))
    return (Q * sig) @ W.T, Q, sig


def gaps(sig):
    """Smallest distance of each singular value to its neighbours."""
    s = np.asarray(sig, np.float64)
    out = np.empty(len(s) - 1)
    for j in range(len(s) - 1):
        lo = s[j] - s[j + 1]
        hi = s[j - 1] - s[j] if j > 0 else np.inf
        out[j] = min(lo, hi)
    return out


def deim_margin(Xi, rows):
    """Smallest ratio, over the DEIM steps, between the largest |residual| and the
    next one: a ratio near 1 means two rows are nearly tied and either is valid."""
    worst = np.inf
    for j in range(Xi.shape[1]):
        xj = Xi[:, j]
        if j == 0:
            res = np.abs(xj)
        else:
            c = np.linalg.solve(Xi[rows[:j], :j], xj[rows[:j]])
            res = np.abs(xj - Xi[:, :j] @ c)
        top2 = np.sort(res)[-2:]
        worst = min(worst, top2[1] / max(top2[0], 1e-300))
    return worst


@pytest.mark.parametrize("shape", [(300, 500), (500, 300), (64, 2000)])
def test_pod_recovers_a_planted_spectrum(P, shape):
    M, K = shape
    sig = 2.0 ** -np.arange(40.0)
    S, Q, _ = planted(11 + M, M, K, sig)
    Xi, s, res, used = P.lrnr_pod(dev(S.T), 16, n_iter=4)
    assert used == 16
    Xo, so = D.pod_basis(S, 16)
    assert np.allclose(s.cpu().numpy(), so, rtol=1e-12, atol=0)
    Xg = Xi.cpu().numpy().T
    assert np.max(np.abs(Xg - Xo)) < 1e-11, np.max(np.abs(Xg - Xo))
    assert np.allclose(np.abs(Xg.T @ Q[:, :16]), np.eye(16), atol=1e-11)
    assert np.all(res.cpu().numpy() < 1e-13)


def test_pod_of_lrnr_snapshots_matches_the_svd(P):
    """Hidden states of an LRNR on the paper's snapshot design (12 points x 9
    perturbations x 8 coefficient draws): singular values to 1e-10 (relative to
    sigma_1), each mode to within its gap-conditioned accuracy, and the span of the
    leading modes to 1e-9."""
    g = synth.rng(21)
    net = synth.make_net(g, L=3, M=256, r=16)
    xs, ts = synth.snapshot_design(g, 8)
    draws = g.uniform(0.5, 1.5, (8, sum(net.r)))
    S = np.concatenate([lrnr64.hidden_states(net, s, xs, ts, 1) for s in draws], axis=1)
    n = 16
    Xi, s, res, used = P.lrnr_pod(dev(S.T), n, n_iter=30)
    Xo, so = D.pod_basis(S, n + 1)
    assert used == n
    sg = s.cpu().numpy()
    assert np.max(np.abs(sg - so[:n])) <= 1e-10 * so[0]
    Xg = Xi.cpu().numpy().T
    gp = gaps(so)
    for j in range(n):
        bound = 1e-12 * so[0] / gp[j] + 1e-12
        assert np.linalg.norm(Xg[:, j] - Xo[:, j]) <= bound, (j, np.linalg.norm(Xg[:, j] - Xo[:, j]), bound)
    # span of the leading 12 modes (well separated from the rest)
    proj = Xo[:, :12] @ (Xo[:, :12].T @ Xg[:, :12])
    assert np.linalg.norm(Xg[:, :12] - proj) < 1e-9
    assert np.all(res.cpu().numpy() < 1e-9)


@pytest.mark.parametrize("shape", [(256, 16, "pod"), (256, 32, "gauss"), (4000, 5, "gauss"),
                                   (97, 13, "gauss"), (33, 32, "gauss")])
def test_deim_rows_match_the_oracle(P, shape):
    M, n, kind = shape
    g = synth.rng(40 + M + n)
    if kind == "pod":
        S = g.standard_normal((M, 3 * n)) * np.exp(-0.25 * np.arange(3 * n))
        Xi, _ = D.pod_basis(S, n)
    else:
        Xi = g.standard_normal((M, n))
    ro = D.deim_rows(Xi)
    assert deim_margin(Xi, ro) > 1 + 1e-9
    rg = P.lrnr_deim_rows(dev(Xi.T)).cpu().numpy()
    assert np.array_equal(rg, ro), (rg, ro)


def test_deim_reports_dependent_columns_and_nan(P):
    g = synth.rng(50)
    Xi = g.standard_normal((40, 4))
    Xi[:, 3] = 2.0 * Xi[:, 1] - Xi[:, 0]
    with pytest.raises(P.LrnrError) as e:
        P.lrnr_deim_rows(dev(Xi.T))
    assert e.value.status == 4      # LRNR_ESINGULAR
    Xi[5, 2] = np.nan
    with pytest.raises(P.LrnrError) as e:
        P.lrnr_deim_rows(dev(Xi[:, :3].T))
    assert e.value.status in (4, 8)
    with pytest.raises(P.LrnrError):
        P.lrnr_deim_rows(dev(np.zeros((40, 33)).T))   # more than 32 columns


def test_pod_rank_cut_and_small_shapes(P):
    S, Q, _ = planted(60, 50, 70, [5.0, 1.0, 0.2])
    Xi, s, _, used = P.lrnr_pod(dev(S.T), 8, n_iter=3, tol=1e-10)
    assert used == 3
    Xg = Xi.cpu().numpy().T
    assert np.allclose(np.abs(Xg.T @ Q), np.eye(3), atol=1e-12)
    # K < n_modes: at most K modes
    g = synth.rng(61)
    S2 = g.standard_normal((30, 4))
    Xi2, s2, _, used2 = P.lrnr_pod(dev(S2.T), 10, n_iter=2, tol=0.0)
    Xo2, so2 = D.pod_basis(S2, 10)
    assert used2 == 4
    assert np.allclose(s2.cpu().numpy(), so2, rtol=1e-12)
    assert np.max(np.abs(Xi2.cpu().numpy().T - Xo2)) < 1e-12
    # M = 1 (a single row)
    Xi3, s3, _, used3 = P.lrnr_pod(dev(np.array([[3.0, -4.0]]).T), 1, n_iter=1)
    assert used3 == 1 and abs(s3.item() - 5.0) < 1e-14 and Xi3.item() == 1.0
    with pytest.raises(P.LrnrError):
        P.lrnr_pod(dev(S.T), 33)


@pytest.mark.parametrize("rhat", [6, 10])
def test_fastlrnr_with_deim_matches_the_oracle(P, rhat):
    """Layer by layer: the oracle's snapshots at the standard design go to both
    sides; the GPU selects with POD + DEIM and installs the reduced layers; the
    FastLRNR loss and gradients then match the oracle's FastLRNR built from the
    oracle's own POD + DEIM (rows identical)."""
    g = synth.rng(70 + rhat)
    net = synth.make_net(g, L=3, M=96, r=16)
    bt = as_f32_batch(synth.make_batch(g, net, 600, 60, 30, 5.0, 1.0, 2.0))
    xs, ts = synth.snapshot_design(g, 8)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    rows_o, Xis_o = [], []
    for l in range(net.L):
        S = lrnr64.hidden_states(net, bt.s[0], xs, ts, l)
        ro, Xo, _, used = D.pod_deim(S, rhat, tol=1e-12)
        assert used == rhat and deim_margin(Xo, ro) > 1 + 1e-6
        rg, Xg, used_g, _ = P.fastlrnr_select_rows_deim(model, l, dev(S.T), rhat, n_iter=30,
                                                        tol=1e-12)
        assert used_g == rhat
        assert np.array_equal(rg.cpu().numpy(), ro), l
        rows_o.append(ro)
        Xis_o.append(Xo)
    fnet = lrnr64.make_fast(net, rows_o, Xis_o)
    db = P.DeviceBatch.from_host(bt)
    lo, ds, dbb = P.lrnr_residual_grad(model, "fast", "fp32", db)
    ro_, rs, rb = lrnr64.residual_grad(fnet, bt, "fast")
    assert rel(lo.cpu(), ro_) < 1e-5
    assert rel(ds.cpu(), rs) < 1e-5, rel(ds.cpu(), rs)
    assert rel(dbb.cpu(), rb) < 1e-5, rel(dbb.cpu(), rb)
    assert P.lrnr_last_device_status(model) == 0
