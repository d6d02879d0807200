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
    on the same device buffers (s, Adam moments, step counter, loss).

    ``copy_in`` / ``copy_out``: optional ``(dst, src)`` tensor pairs copied before /
    after the steps inside the same graph, e.g. a batch staged in pinned host memory
    going to the device buffers the batch views, and ``s`` and the loss coming back
    to pinned host memory, so that one replay is a whole host-to-host step.  Each pair
    is copied by the library's copy kernel (``lrnr_copy_pinned``: loads and stores
    through the unified address space, host bytes read uncached), so a replay sees
    what the host wrote to a pinned source before it."""

    def __init__(self, model, batch, s, m, v, step, n_steps=1, form="fast", prec="fp32",
                 loss_out=None, copy_in=(), copy_out=(), **adam):
        B.lrnr_reserve(model, batch.n_points, batch.n_inst)
        self.args = (model, form, prec, batch, s, m, v, step)
        self.kw = dict(n_steps=n_steps, loss_out=loss_out, **adam)
        self.copy_in, self.copy_out = tuple(copy_in), tuple(copy_out)
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):          # warm-up outside the graph
            self._body()
        torch.cuda.current_stream().wait_stream(stream)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            self._body()

    def _body(self):
        for dst, src in self.copy_in:
            B.lrnr_copy_pinned(dst, src)
        B.spinprop_step(*self.args, **self.kw)
        for dst, src in self.copy_out:
            B.lrnr_copy_pinned(dst, src)

    def replay(self):
        self.graph.replay()
