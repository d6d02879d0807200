"""Pins of the oracle's FastLRNR and EIM: identities and properties fixed by Eq. 2.6-2.8."""
import itertools

import numpy as np
import pytest

import synth
from oracle import eim64 as E
from oracle import lrnr64 as O
from tests.oracle_helpers import relerr


def case(seed=9, L=3, M=10, r=3, r1=None, mu=(5.0, 1.0, 2.0), n_int=30, n_ic=7, n_bc=5):
    g = synth.rng(seed)
    net = synth.make_net(g, L=L, M=M, r=r, r1=r1)
    bt = synth.make_batch(g, net, n_int, n_ic, n_bc, *mu)
    return g, net, bt


def test_fast_equals_full_when_every_row_is_kept():
    _, net, bt = case()
    I = np.eye(net.M)
    fnet = O.make_fast(net, [np.arange(net.M)] * net.L, [I] * net.L)
    inst = bt.instance(0)
    uf, _ = O.full_forward(net, inst["s"], inst["x_int"], inst["t_int"])
    uh, _ = O.fast_forward(fnet, inst["s"], inst["x_int"], inst["t_int"])
    assert relerr(uh, uf) < 1e-14
    for loss in ("mse", "l1"):
        lf, dsf, dbf = O.instance_loss_grad(O.full_forward, O.full_backward, net, inst, loss)
        lh, dsh, dbh = O.instance_loss_grad(O.fast_forward, O.fast_backward, fnet, inst, loss)
        assert abs(lf - lh) <= 1e-14 * abs(lf)
        assert relerr(dsh, dsf) < 1e-13
        assert relerr(dbh, dbf) < 1e-13


def test_fast_equals_full_with_greedy_rows_on_a_spanning_snapshot_set():
    g, net, bt = case(seed=4)
    xs, ts = g.uniform(0, 2 * np.pi, 60), g.uniform(0, 1, 60)
    rows, Xis = [], []
    for l in range(net.L):
        S = O.hidden_states(net, bt.s[0], xs, ts, l)
        p, Xi, used = E.eim_greedy(S, net.M)
        assert used == net.M and sorted(p.tolist()) == list(range(net.M))
        rows.append(p)
        Xis.append(Xi)
    fnet = O.make_fast(net, rows, Xis)
    inst = bt.instance(0)
    lf, dsf, dbf = O.instance_loss_grad(O.full_forward, O.full_backward, net, inst)
    lh, dsh, dbh = O.instance_loss_grad(O.fast_forward, O.fast_backward, fnet, inst)
    assert abs(lf - lh) <= 1e-10 * abs(lf)
    assert relerr(dsh, dsf) < 1e-9
    assert relerr(dbh, dbf) < 1e-9


def test_fast_agrees_with_full_at_the_snapshot_points():
    """When layer l's snapshots are the exact states at K <= rh points, the reduced
    network reproduces u exactly there (the agreement the paper shows in Fig. 2)."""
    g, net, bt = case(seed=12, L=4, M=24, r=4)
    K, rh = 5, 8
    xs, ts = g.uniform(0, 2 * np.pi, K), g.uniform(0, 1, K)
    s = bt.s[0]
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, used = E.eim_greedy(O.hidden_states(net, s, xs, ts, l), rh, tol=1e-10)
        assert used == K
        rows.append(p)
        Xis.append(Xi)
    fnet = O.make_fast(net, rows, Xis)
    uf, _ = O.full_forward(net, s, xs, ts)
    uh, _ = O.fast_forward(fnet, s, xs, ts)
    assert relerr(uh[:, 0], uf[:, 0]) < 1e-12
    # away from the samples the reduced network is only an approximation
    x2, t2 = g.uniform(0, 2 * np.pi, 50), g.uniform(0, 1, 50)
    assert relerr(O.fast_forward(fnet, s, x2, t2)[0][:, 0], O.full_forward(net, s, x2, t2)[0][:, 0]) > 1e-8


def test_fast_gradient_matches_central_differences():
    g, net, bt = case(seed=6, L=3, M=12, r=3)
    xs, ts = g.uniform(0, 2 * np.pi, 40), g.uniform(0, 1, 40)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _ = E.eim_greedy(O.hidden_states(net, bt.s[0], xs, ts, l), 6)
        rows.append(p)
        Xis.append(Xi)
    fnet = O.make_fast(net, rows, Xis)
    inst = bt.instance(0)
    _, ds, db = O.instance_loss_grad(O.fast_forward, O.fast_backward, fnet, inst)
    h = 1e-6
    fd = np.zeros_like(ds)
    for k in range(ds.shape[0]):
        sp, sm = dict(inst), dict(inst)
        sp["s"] = inst["s"].copy()
        sm["s"] = inst["s"].copy()
        sp["s"][k] += h
        sm["s"][k] -= h
        fd[k] = (O.instance_loss_grad(O.fast_forward, O.fast_backward, fnet, sp)[0]
                 - O.instance_loss_grad(O.fast_forward, O.fast_backward, fnet, sm)[0]) / (2 * h)
    assert relerr(ds, fd) < 1e-7
    # bias gradient: perturb bhat (= b at the selected rows) of each layer
    off = np.cumsum([0] + [b.shape[0] for b in net.b])
    for l in range(net.L):
        for j, row in enumerate(fnet.rows[l]):
            bp, bm = [x.copy() for x in fnet.bh], [x.copy() for x in fnet.bh]
            bp[l][j] += h
            bm[l][j] -= h
            fp = O.FastNet(net, fnet.rows, fnet.Uh, bp, fnet.Vh)
            fm = O.FastNet(net, fnet.rows, fnet.Uh, bm, fnet.Vh)
            fdb = (O.instance_loss_grad(O.fast_forward, O.fast_backward, fp, inst)[0]
                   - O.instance_loss_grad(O.fast_forward, O.fast_backward, fm, inst)[0]) / (2 * h)
            assert abs(db[off[l] + row] - fdb) < 1e-7 * max(1e-3, abs(fdb)) + 1e-9
    # rows that were not selected carry no bias gradient
    for l in range(net.L):
        mask = np.ones(net.M, bool)
        mask[fnet.rows[l]] = False
        assert np.all(db[off[l]:off[l + 1]][mask] == 0.0)


def test_fast_network_of_x_minus_beta_t_has_zero_convection_residual():
    beta = 7.0
    g, net, bt = case(seed=30, L=3, M=16, r=4, r1=1, mu=(beta, 0.0, 0.0))
    net.V[0] = np.array([[1.1], [-1.1 * beta]])
    xs, ts = g.uniform(0, 2 * np.pi, 30), g.uniform(0, 1, 30)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _ = E.eim_greedy(O.hidden_states(net, bt.s[0], xs, ts, l), 6)
        rows.append(p)
        Xis.append(Xi)
    fnet = O.make_fast(net, rows, Xis)
    u, _ = O.fast_forward(fnet, bt.s[0], bt.x_int, bt.t_int)
    R = O.cdr_residual(u[:, 0], u[:, 1], u[:, 2], u[:, 3], beta, 0.0, 0.0)
    assert np.max(np.abs(R)) < 1e-12 * max(1.0, beta * np.max(np.abs(u[:, 2])))
    assert np.max(np.abs(u[:, 2])) > 1e-5


# --------------------------------------------------------------------------- EIM

def test_eim_on_scaled_unit_vectors_picks_rows_by_decreasing_magnitude():
    M = 9
    idx = [4, 0, 7, 2, 5]
    c = [0.3, -2.5, 1.2, 0.05, -0.9]
    S = np.zeros((M, len(idx)))
    for k, (i, ck) in enumerate(zip(idx, c)):
        S[i, k] = ck
    rows, Xi, used = E.eim_greedy(S, 5)
    order = np.argsort(-np.abs(c), kind="stable")
    assert used == 5
    assert rows.tolist() == [idx[k] for k in order]
    assert np.array_equal(Xi, np.eye(M)[:, rows])


def test_eim_structure_on_random_snapshots():
    g = synth.rng(44)
    S = g.normal(size=(30, 50))
    rows, Xi, used = E.eim_greedy(S, 12)
    assert used == 12 and len(set(rows.tolist())) == 12
    T = Xi[rows, :]
    assert np.array_equal(np.diag(T), np.ones(12))          # exactly 1: x / x
    assert np.array_equal(np.triu(T, 1), np.zeros((12, 12)))  # exactly 0 above the diagonal
    # the interpolant reproduces its values at the selected rows exactly (up to the solve)
    v = g.normal(size=30)
    w = E.interpolate(Xi, rows, v)
    assert np.max(np.abs(w[rows] - v[rows])) < 1e-12


def test_eim_interpolates_spanned_snapshots_and_stops_early():
    g = synth.rng(45)
    S = g.normal(size=(20, 4)) @ g.normal(size=(4, 15))   # rank 4
    rows, Xi, used = E.eim_greedy(S, 10, tol=1e-9)
    assert used == 4
    assert relerr(E.interpolate(Xi, rows, S), S) < 1e-12


def test_eim_tie_break_lowest_index():
    S = np.array([[1.0, -3.0, 3.0], [3.0, 1.0, 0.5], [-3.0, 0.2, 0.1]])
    rows, Xi, used = E.eim_greedy(S, 1)
    # columns 0, 1, 2 all have max |.| = 3 -> column 0; in column 0 rows 1 and 2 tie -> row 1
    assert rows.tolist() == [1]
    assert np.array_equal(Xi[:, 0], S[:, 0] / 3.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eim_greedy_matches_brute_force_replay(seed):
    """Replay the greedy rule without the incremental update: at step j the residual
    is S minus its interpolant on the rows chosen so far (fresh solve), and the
    chosen column / row must be the max-abs ones (lowest index among ties)."""
    g = synth.rng(100 + seed)
    M, K, rh = 7, 11, 6
    S = g.normal(size=(M, K))
    rows, Xi, used = E.eim_greedy(S, rh)
    assert used == rh
    for j in range(rh):
        if j == 0:
            Rj = S
        else:
            P = rows[:j]
            basis = Xi[:, :j]
            Rj = S - basis @ np.linalg.solve(basis[P, :], S[P, :])
        e = np.max(np.abs(Rj), axis=0)
        kstar = int(np.argmax(e))
        assert np.isclose(np.max(e), e[kstar])
        assert rows[j] == int(np.argmax(np.abs(Rj[:, kstar])))
        assert np.allclose(Xi[:, j], Rj[:, kstar] / Rj[rows[j], kstar], rtol=1e-10, atol=1e-12)
    # exhaustive check on the first step: no (row, column) pair beats the pivot
    best = max(((abs(S[i, k]), -k, -i) for i, k in itertools.product(range(M), range(K))))
    assert rows[0] == -best[2]
