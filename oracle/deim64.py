"""FP64 CPU oracle of the DEIM variant of the FastLRNR layer reduction (Sec. 2.2,
Eq. 2.7, with the discrete empirical interpolation method the paper cites beside
EIM).

TEST INFRASTRUCTURE ONLY (see ``oracle/lrnr64.py``).

Eq. 2.7 leaves the basis Xi and the sampling matrix P open.  In the DEIM reading:

  POD basis.  Xi = the n leading left singular vectors of the snapshot matrix S
    (M x K), from its thin SVD S = Q diag(sigma) W^T with sigma descending.  Mode j
    is kept only while sigma_j > tol * sigma_1 (a relative cut; tol = 0 keeps every
    mode with a nonzero singular value).  Singular vectors are fixed only up to
    sign, so each kept column is scaled by +-1 to make its entry of largest
    magnitude (lowest index among exact ties) positive.
  DEIM indices.  p_1 = argmax_i |xi_1(i)|.  For j = 2..n: interpolate xi_j through
    the rows chosen so far with the first j-1 columns,
        c = (P_{j-1}^T Xi_{j-1})^{-1} P_{j-1}^T xi_j,
    and take p_j = argmax_i |xi_j(i) - (Xi_{j-1} c)(i)| (lowest index among exact
    ties).  The residual vanishes on the rows already chosen, so the rows are
    distinct and P^T Xi is invertible.  A residual whose largest magnitude is at most
    1e-12 of the column's own largest entry (rounding level: the column lies in the
    span of the earlier ones) stops the selection with an error.

Then the reduced layer is Eq. 2.7 with this (Xi, P).  P^T Xi is invertible but, unlike
the EIM basis, not triangular, so V-hat takes a general solve
(``lrnr64.reduce_layer`` solves with partial pivoting).
"""
from __future__ import annotations

import numpy as np


DEPENDENT = 1e-12   # relative residual at which a basis column counts as dependent


def canonical_signs(Xi: np.ndarray) -> np.ndarray:
    """Scale each column by +-1 so that its entry of largest magnitude (the first
    such entry) is positive."""
    Xi = np.array(Xi, dtype=np.float64, copy=True)
    for j in range(Xi.shape[1]):
        i = int(np.argmax(np.abs(Xi[:, j])))
        if Xi[i, j] < 0.0:
            Xi[:, j] = -Xi[:, j]
    return Xi


def pod_basis(S: np.ndarray, n: int, tol: float = 0.0):
    """The n leading POD modes of the snapshot matrix S (M x K): returns
    (Xi (M, n_kept), sigma (n_kept,)), n_kept <= min(n, M, K)."""
    S = np.asarray(S, dtype=np.float64)
    Q, sig, _ = np.linalg.svd(S, full_matrices=False)
    n = min(int(n), sig.shape[0])
    kept = 0
    while kept < n and sig[kept] > tol * sig[0] and sig[kept] > 0.0:
        kept += 1
    return canonical_signs(Q[:, :kept]), sig[:kept].copy()


def deim_rows(Xi: np.ndarray) -> np.ndarray:
    """DEIM index selection on the columns of Xi (M x n, linearly independent):
    returns the rows (int64, (n,)) in the order they are chosen."""
    Xi = np.asarray(Xi, dtype=np.float64)
    M, n = Xi.shape
    rows: list[int] = []
    for j in range(n):
        xj = Xi[:, j]
        if j == 0:
            res = xj
        else:
            P = np.array(rows, dtype=np.int64)
            c = np.linalg.solve(Xi[P, :j], xj[P])
            res = xj - Xi[:, :j] @ c
        p = int(np.argmax(np.abs(res)))       # first occurrence: lowest index among ties
        if p in rows or not np.abs(res[p]) > DEPENDENT * np.max(np.abs(xj)):
            raise np.linalg.LinAlgError("DEIM: the basis columns are not independent")
        rows.append(p)
    return np.array(rows, dtype=np.int64)


def pod_deim(S: np.ndarray, rh: int, tol: float = 0.0):
    """POD basis of S and its DEIM rows: returns (rows, Xi, sigma, rh_used)."""
    Xi, sig = pod_basis(S, rh, tol)
    rows = deim_rows(Xi) if Xi.shape[1] else np.zeros(0, dtype=np.int64)
    return rows, Xi, sig, Xi.shape[1]
