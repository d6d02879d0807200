"""Splitting a batch of PDE instances across ranks.

Instances are independent (each has its own s, Adam state and loss), so N ranks
each take a contiguous block of instances and no data-path collective is needed;
the bases are replicated read-only.  Only timing uses a collective (max over ranks).
"""
from __future__ import annotations

import numpy as np


def instance_range(n_inst: int, world: int, rank: int):
    """Contiguous block [lo, hi) of instances owned by ``rank`` (sizes differ by <= 1)."""
    base, extra = divmod(n_inst, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def subset(batch, lo: int, hi: int):
    """Host batch (fields as in ``synth.Batch``) restricted to instances [lo, hi)."""
    def cut(off, *arrs):
        a, b = int(off[lo]), int(off[hi])
        return (off[lo:hi + 1] - off[lo],) + tuple(x[a:b] for x in arrs)
    io, xi, ti = cut(batch.int_off, batch.x_int, batch.t_int)
    co, xc = cut(batch.ic_off, batch.x_ic)
    bo, tb = cut(batch.bc_off, batch.t_bc)
    return type(batch)(beta=batch.beta[lo:hi], nu=batch.nu[lo:hi], rho=batch.rho[lo:hi],
                       s=batch.s[lo:hi], int_off=np.asarray(io), ic_off=np.asarray(co),
                       bc_off=np.asarray(bo), x_int=xi, t_int=ti, x_ic=xc, t_bc=tb)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank scalar (timing); identity without a process group."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
