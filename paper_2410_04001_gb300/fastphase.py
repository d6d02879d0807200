"""The fast phase of FastLRNR (Sec. 3.2, Eq. 3.6-3.7; Sec. 4): build the reduced
network from exact-LRNR snapshots at a sparse sample set X, train the coefficients
s of one PDE instance through the reduced network with the l1 physics loss and the
l1 locality term, and return the solution on the full-width LRNR with the trained
coefficients, u_FASTSOL = u_LRNR(.; s_fast).

This module only sequences calls of the C ABI (``liblrnr.so``); every step runs in
its kernels: snapshots and the EIM greedy in FP64 (``lrnr_snapshots``,
``fastlrnr_select_rows``; or the POD basis and DEIM rows, ``lrnr_pod`` and
``lrnr_deim_rows``), the SPInProp Adam steps (``spinprop_step`` with the l1
loss and the locality term), and the full-width evaluation (``lrnr_residual``).
"""
from __future__ import annotations

import torch

from . import binding as B


def build_reduced(model: B.Model, x, t, s_draws, rhat: int, tol: float = 0.0, stream=None,
                  method: str = "eim", n_iter: int = 30):
    """Select the rows of every hidden layer from the exact-LRNR states at the points
    (x, t) (device FP64 vectors, the sample set X and its perturbations) for each
    coefficient vector in ``s_draws`` (n_s x sum_r); installs the reduced layers in
    ``model`` and returns, per layer, the rows and the number kept.

    ``method="eim"``: the greedy EIM of ``fastlrnr_select_rows`` (``tol`` is its
    absolute stopping level).  ``method="deim"``: POD basis by ``lrnr_pod``
    (``n_iter`` subspace iterations; ``tol`` is the relative singular-value cut,
    1e-10 when 0 is passed) and DEIM rows by ``lrnr_deim_rows``."""
    if method not in ("eim", "deim"):
        raise ValueError(f"unknown selection method {method!r}")
    out = []
    for layer in range(model.L):
        S = B.lrnr_snapshots(model, layer, x, t, s_draws, stream=stream)
        if method == "eim":
            rows, _, used = B.fastlrnr_select_rows(model, layer, S, rhat, tol, stream=stream)
        else:
            rows, _, used, _ = B.fastlrnr_select_rows_deim(model, layer, S, rhat, n_iter=n_iter,
                                                           tol=tol if tol > 0 else 1e-10,
                                                           stream=stream)
        out.append((rows, used))
    return out


def fast_phase(model: B.Model, batch_X: B.DeviceBatch, n_steps: int, lr: float = 1e-3,
               lambda_loc: float = 0.0, s_anchor=None, loss_out=None, prec: str = "fp32",
               stream=None):
    """``n_steps`` Adam steps on the coefficients of ``batch_X`` (its ``s`` is copied,
    not modified) minimising the fast loss of Eq. 3.6 plus lambda_loc times the
    locality term of Eq. 3.7 (anchor ``s_anchor``, the coefficients the phase starts
    from when omitted).  ``prec``: "fp32" (FP32 kernel) or "bf16" / "bf16x3" (the
    reduced network on the tensor cores).  Returns the trained coefficients s_fast
    (device, FP32)."""
    s = batch_X.s.clone()
    anchor = s.clone() if s_anchor is None else s_anchor
    m = torch.zeros_like(s)
    v = torch.zeros_like(s)
    step = torch.zeros(1, dtype=torch.int64, device=s.device)
    B.spinprop_step(model, "fast", prec, batch_X, s, m, v, step, n_steps=n_steps, lr=lr,
                    lambda_loc=lambda_loc, s_anchor=anchor, loss="l1", loss_out=loss_out,
                    stream=stream)
    return s


def fast_solution(model: B.Model, batch_eval: B.DeviceBatch, s_fast, prec: str = "fp32",
                  stream=None):
    """u_FASTSOL at the interior points of ``batch_eval``: the full-width LRNR with the
    coefficients s_fast (returns u and the CDR residual at those points)."""
    out = B.lrnr_residual(model, "full", prec, batch_eval.with_s(s_fast), stream=stream)
    return out
