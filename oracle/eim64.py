"""FP64 CPU oracle of the EIM row selection behind FastLRNR (Sec. 2.2, Eq. 2.7).

TEST INFRASTRUCTURE ONLY (see ``oracle/lrnr64.py``).

Classic greedy empirical interpolation, incremental (Newton) form.  Given a
snapshot matrix ``S`` (M x K, columns are hidden-state vectors of the exact LRNR):

    R <- S
    for j = 1..rh:
        e_k = max_i |R_ik|                      (per column)
        k*  = argmax_k e_k                      (lowest k among exact ties)
        stop if e_k* <= tol                     (then rh_used = j - 1)
        p_j = argmax_i |R_i,k*|                 (lowest i among exact ties)
        xi_j = R[:, k*] / R[p_j, k*]            (IEEE division)
        R <- R - xi_j (outer) R[p_j, :]         (a product, then a difference: no FMA)

``Xi = [xi_1 .. xi_rh]`` and ``P = (p_1 .. p_rh)``; ``P^T Xi`` is unit lower
triangular, so the interpolation ``Xi (P^T Xi)^{-1} P^T`` exists.  The paper does
not fix the basis source, the tie-breaks, nor the stopping rule; the choices
above are this library's reading.
"""
from __future__ import annotations

import numpy as np


def eim_greedy(S: np.ndarray, rh: int, tol: float = 0.0):
    """Returns (rows int64 (rh_used,), Xi (M, rh_used), rh_used)."""
    R = np.array(S, dtype=np.float64, copy=True)
    M, K = R.shape
    rows, cols = [], []
    for _ in range(min(rh, M)):
        e = np.max(np.abs(R), axis=0)
        k = int(np.argmax(e))            # first occurrence: lowest index among ties
        if not (e[k] > tol):
            break
        p = int(np.argmax(np.abs(R[:, k])))
        xi = R[:, k] / R[p, k]
        prod = np.multiply.outer(xi, R[p, :])   # rounded products
        R = R - prod                             # rounded differences
        rows.append(p)
        cols.append(xi)
    rh_used = len(rows)
    Xi = np.stack(cols, axis=1) if rh_used else np.zeros((M, 0))
    return np.array(rows, dtype=np.int64), Xi, rh_used


def interpolate(Xi: np.ndarray, rows: np.ndarray, v: np.ndarray) -> np.ndarray:
    """EIM interpolant ``Xi (P^T Xi)^{-1} P^T v`` of a vector (or columns) ``v``."""
    rows = np.asarray(rows, dtype=np.int64)
    coef = np.linalg.solve(Xi[rows, :], v[rows])
    return Xi @ coef
