"""The adjoint kernels behind ``torch.autograd`` (sparse physics-informed backprop).

``lrnr_loss(s, model, batch)`` returns the per-instance physics-informed loss
(Eq. 3.5 or Eq. 3.6) of the LRNR or FastLRNR with coefficients ``s`` and is
differentiable in ``s``.  The forward pass runs ``lrnr_residual_grad``, whose fused
kernel already produces dL/ds by the hand-written adjoint (each layer's
pre-activation is rebuilt from its stored rank-r input instead of keeping M-wide
activations); backward only scales it by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import binding as B


class LRNRLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, model, batch, form, prec, loss, w):
        s = s.detach().contiguous()
        bt = batch.with_s(s)
        lo, ds, _ = B.lrnr_residual_grad(model, form, prec, bt, loss=loss, w=w, want_db=False)
        ctx.save_for_backward(ds)
        return lo

    @staticmethod
    def backward(ctx, grad_loss):
        ds, = ctx.saved_tensors
        return grad_loss[:, None] * ds, None, None, None, None, None, None


def lrnr_loss(s, model, batch, form="fast", prec="fp32", loss="mse", w=None):
    """Per-instance loss, differentiable in ``s`` (shape (n_inst, sum_r), float32, CUDA)."""
    return LRNRLoss.apply(s, model, batch, form, prec, loss, w)
