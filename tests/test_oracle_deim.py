"""Pins of the oracle's DEIM variant (POD basis + discrete empirical interpolation
indices, Sec. 2.2 Eq. 2.7): each check is fixed by the mathematics, not by the
oracle's own formulas."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import deim64 as D
from oracle import eim64 as E
from oracle import lrnr64 as O
from tests.oracle_helpers import relerr


def orthonormal(g, n, k):
    q, _ = np.linalg.qr(g.standard_normal((n, k)))
    return q


def planted(g, M=40, K=60, sig=(8.0, 4.0, 2.0, 1.0, 0.5, 0.25, 0.125, 0.0625)):
    sig = np.asarray(sig)
    Q, W = orthonormal(g, M, len(sig)), orthonormal(g, K, len(sig))
    return Q, sig, (Q * sig) @ W.T


def test_pod_recovers_a_planted_spectrum_and_truncates_at_its_rank():
    g = synth.rng(301)
    Q, sig, S = planted(g)
    Xi, s = D.pod_basis(S, 5)
    assert np.allclose(s, sig[:5], rtol=1e-13, atol=0)
    # the same subspace, column by column up to sign
    assert np.allclose(np.abs(Xi.T @ Q[:, :5]), np.eye(5), atol=1e-12)
    # the sign convention: the largest-magnitude entry of each column is positive
    for j in range(5):
        i = np.argmax(np.abs(Xi[:, j]))
        assert Xi[i, j] > 0
    # rank 8: asking for 12 modes keeps only the 8 above the relative cut
    Xi12, s12 = D.pod_basis(S, 12, tol=1e-10)
    assert Xi12.shape == (40, 8) and s12.shape == (8,)


@pytest.mark.parametrize("shape", [(30, 50), (50, 30)])
def test_pod_modes_are_eigenvectors_of_the_gram_matrix_and_optimal(shape):
    """Left singular vectors of S are the eigenvectors of S S^T (eigenvalues
    sigma^2), and the rank-n projection error is the sum of the discarded
    eigenvalues (Eckart-Young), both checked with a symmetric eigen-solver."""
    g = synth.rng(302)
    S = g.standard_normal(shape) * np.exp(-0.3 * np.arange(shape[1]))
    n = 7
    Xi, s = D.pod_basis(S, n)
    G = S @ S.T
    assert np.linalg.norm(G @ Xi - Xi * s**2) <= 1e-12 * np.linalg.norm(G)
    lam = np.sort(np.linalg.eigvalsh(G))[::-1]
    err = np.linalg.norm(S - Xi @ (Xi.T @ S)) ** 2
    assert abs(err - lam[n:].sum()) <= 1e-10 * lam[0]
    assert np.allclose(Xi.T @ Xi, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_deim_rows_are_the_pivots_of_lu_with_partial_pivoting(seed):
    """Step j of DEIM maximises |column j of the Schur complement| over the rows not
    yet chosen: exactly the row that Gaussian elimination with partial pivoting
    (LAPACK getrf) swaps in at step j."""
    g = synth.rng(310 + seed)
    M, n = 25 + 7 * seed, 4 + seed
    Xi = g.standard_normal((M, n))
    _, piv = scipy.linalg.lu_factor(Xi)
    perm = np.arange(M)
    for i in range(n):
        perm[i], perm[piv[i]] = perm[piv[i]], perm[i]
    assert np.array_equal(D.deim_rows(Xi), perm[:n])


def test_deim_on_unit_vectors_picks_their_rows_in_order():
    M = 12
    order = [7, 2, 11, 0, 5]
    Xi = np.zeros((M, len(order)))
    for j, i in enumerate(order):
        Xi[i, j] = 1.0 if j % 2 == 0 else -1.0
    assert np.array_equal(D.deim_rows(Xi), order)


def test_deim_tie_break_lowest_index():
    Xi = np.array([[1.0, 0.0], [-1.0, 1.0], [0.5, -1.0], [0.0, 0.0]])
    # |xi_1| ties at rows 0 and 1 -> 0; then the residual of xi_2 is
    # xi_2 - xi_1 * 0 = xi_2, whose magnitude ties at rows 1 and 2 -> 1
    assert np.array_equal(D.deim_rows(Xi), [0, 1])


def test_deim_interpolates_the_span_and_obeys_the_deim_error_bound():
    """The DEIM projector Xi (P^T Xi)^{-1} P^T reproduces every vector of span(Xi);
    its inverse block obeys ||(P^T Xi)^{-1}||_2 <= (1 + sqrt(2M))^{n-1} / ||xi_1||_inf
    (the DEIM bound for an orthonormal basis)."""
    g = synth.rng(320)
    M, n = 60, 9
    S = g.standard_normal((M, 80)) * np.exp(-0.2 * np.arange(80))
    rows, Xi, sig, used = D.pod_deim(S, n)
    assert used == n and len(set(rows.tolist())) == n
    f = Xi @ g.standard_normal(n)
    assert relerr(E.interpolate(Xi, rows, f), f) < 1e-13
    inv = np.linalg.norm(np.linalg.inv(Xi[rows, :]), 2)
    assert inv <= (1 + np.sqrt(2 * M)) ** (n - 1) / np.max(np.abs(Xi[:, 0]))
    # sign and scale of each column do not move the rows
    scale = g.choice([-3.0, -0.5, 0.25, 2.0], n)
    assert np.array_equal(D.deim_rows(Xi * scale), rows)
    # relabelling the rows relabels the selection
    perm = g.permutation(M)
    inv_perm = np.argsort(perm)
    assert np.array_equal(D.deim_rows(Xi[perm, :]), inv_perm[rows])


def test_fast_network_with_deim_agrees_with_full_at_the_snapshot_points():
    """With the snapshots of every layer the exact states at K <= rh points, the POD
    basis spans them, so the DEIM-reduced network reproduces u there (Fig. 2's
    agreement at the sample set), and only approximates it elsewhere."""
    g = synth.rng(330)
    net = synth.make_net(g, L=4, M=24, r=4)
    K, rh = 5, 8
    xs, ts = g.uniform(0, 2 * np.pi, K), g.uniform(0, 1, K)
    s = g.uniform(0.5, 1.5, sum(net.r))
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _, used = D.pod_deim(O.hidden_states(net, s, xs, ts, l), rh, tol=1e-10)
        assert used == K
        rows.append(p)
        Xis.append(Xi)
    fnet = O.make_fast(net, rows, Xis)
    uf, _ = O.full_forward(net, s, xs, ts)
    uh, _ = O.fast_forward(fnet, s, xs, ts)
    assert relerr(uh[:, 0], uf[:, 0]) < 1e-12
    x2, t2 = g.uniform(0, 2 * np.pi, 50), g.uniform(0, 1, 50)
    assert relerr(O.fast_forward(fnet, s, x2, t2)[0][:, 0],
                  O.full_forward(net, s, x2, t2)[0][:, 0]) > 1e-8


def test_fast_network_with_deim_on_every_row_is_the_full_network():
    """rh = M with a full-rank snapshot set: the POD basis is a basis of R^M, DEIM
    picks every row once, and the reduced network equals the full one."""
    g = synth.rng(331)
    net = synth.make_net(g, L=3, M=10, r=3)
    s = g.uniform(0.5, 1.5, sum(net.r))
    xs, ts = g.uniform(0, 2 * np.pi, 40), g.uniform(0, 1, 40)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _, used = D.pod_deim(O.hidden_states(net, s, xs, ts, l), net.M)
        assert used == net.M and sorted(p.tolist()) == list(range(net.M))
        rows.append(p)
        Xis.append(Xi)
    fnet = O.make_fast(net, rows, Xis)
    x2, t2 = g.uniform(0, 2 * np.pi, 30), g.uniform(0, 1, 30)
    uf, _ = O.full_forward(net, s, x2, t2)
    uh, _ = O.fast_forward(fnet, s, x2, t2)
    assert relerr(uh, uf) < 1e-10


def test_deim_rejects_a_dependent_column():
    g = synth.rng(340)
    Xi = g.standard_normal((30, 4))
    Xi[:, 3] = 2.0 * Xi[:, 1] - Xi[:, 0]
    with pytest.raises(np.linalg.LinAlgError):
        D.deim_rows(Xi)
    Xi[:, 3] += 1e-9 * g.standard_normal(30)     # independent, if barely
    assert len(set(D.deim_rows(Xi).tolist())) == 4
