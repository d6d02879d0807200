"""CUDA-graph capture of launch-bound loops (the SPInProp fast phase).

A SPInProp step is one kernel (batches whose tiles fit in one round of the grid:
the tile kernel also reduces the gradient and applies Adam) or two (the tile kernel,
then the fixed-order reduction with Adam); at the paper's fast-phase sizes (12
collocation points, a few thousand in batched use) the host launch cost dominates,
so the whole loop of ``n_steps`` steps is captured once and replayed.
"""
from __future__ import annotations

import torch

from . import binding as B


class SpinpropGraph:
    """Captured ``spinprop_step(..., n_steps)``; ``replay()`` runs the steps again
    on the same device buffers (s, Adam moments, step counter, loss)."""

    def __init__(self, model, batch, s, m, v, step, n_steps=1, form="fast", prec="fp32",
                 loss_out=None, **adam):
        B.lrnr_reserve(model, batch.n_points, batch.n_inst)
        self.args = (model, form, prec, batch, s, m, v, step)
        self.kw = dict(n_steps=n_steps, loss_out=loss_out, **adam)
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):          # warm-up outside the graph
            B.spinprop_step(*self.args, **self.kw)
        torch.cuda.current_stream().wait_stream(stream)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            B.spinprop_step(*self.args, **self.kw)

    def replay(self):
        self.graph.replay()
