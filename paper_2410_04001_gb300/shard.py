"""Data-parallel splits of the hot path across ranks (one process per GPU).

Two splits, both from the structure of the loss:

* By instance.  Instances are independent (each has its own s, Adam state and
  loss), so N ranks each take a contiguous block of instances and no data-path
  collective is needed; the bases are replicated read-only.
* By point, within an instance.  The physics-informed loss of Eq. 3.5 is a sum
  over collocation points divided by the point counts, and its gradient is a sum
  over points (Sec. 2.3).  Each rank takes a block of every instance's points of
  every class and evaluates them with the whole instance's counts as the MSE
  denominators (``lrnr_batch.norm``); its loss, dL/ds and dL/db are then partial
  sums, and one sum all-reduce of (loss, dL/ds, dL/db) gives every rank the
  instance's loss and gradient.  The Adam update that follows is replicated.

Only the collective itself (``torch.distributed.all_reduce``) runs outside the
library: the per-rank evaluation and the Adam update are library calls.
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


def instance_counts(batch):
    """(n_inst, 3) int64: each instance's interior points, initial points and
    periodic pairs -- the MSE denominators of Eq. 3.5."""
    return np.stack([np.diff(batch.int_off), np.diff(batch.ic_off), np.diff(batch.bc_off)],
                    axis=1).astype(np.int64)


def point_shard(batch, world: int, rank: int):
    """Rank ``rank``'s share of every instance's points: for each instance and each
    point class (interior, initial, periodic pairs) the contiguous block
    ``instance_range(count, world, rank)`` of that class's points.  Returns the
    host batch of those points (every instance kept, possibly with no points) and
    the whole batch's per-instance counts (``instance_counts``), which are the
    shard's MSE denominators."""
    counts = instance_counts(batch)

    def take(off, *arrs):
        new_off = [0]
        parts = [[] for _ in arrs]
        for i in range(batch.n_inst):
            a, b = int(off[i]), int(off[i + 1])
            lo, hi = instance_range(b - a, world, rank)
            for p, x in zip(parts, arrs):
                p.append(x[a + lo:a + hi])
            new_off.append(new_off[-1] + (hi - lo))
        cat = [np.concatenate(p) if p else np.zeros(0) for p in parts]
        return (np.asarray(new_off, np.int64),) + tuple(cat)

    io, xi, ti = take(batch.int_off, batch.x_int, batch.t_int)
    co, xc = take(batch.ic_off, batch.x_ic)
    bo, tb = take(batch.bc_off, batch.t_bc)
    shard = type(batch)(beta=batch.beta, nu=batch.nu, rho=batch.rho, s=batch.s, int_off=io,
                        ic_off=co, bc_off=bo, x_int=xi, t_int=ti, x_ic=xc, t_bc=tb)
    return shard, counts


def partial_buffers(n_inst: int, sum_r: int, sum_m: int, want_db: bool, device=None, dtype=None):
    """One flat buffer for (loss, dL/ds, dL/db) and its three contiguous views, so
    that the partial sums of a rank go through a single all-reduce."""
    import torch
    dtype = dtype or torch.float32
    n = n_inst * (1 + sum_r + (sum_m if want_db else 0))
    flat = torch.zeros(n, dtype=dtype, device=device)
    loss = flat[:n_inst]
    ds = flat[n_inst:n_inst * (1 + sum_r)].view(n_inst, sum_r)
    db = flat[n_inst * (1 + sum_r):].view(n_inst, sum_m) if want_db else None
    return flat, (loss, ds, db)


def sharded_residual_grad(local_fn, n_inst: int, sum_r: int, sum_m: int, dist, want_db=True,
                          device=None, dtype=None, bufs=None):
    """Loss, dL/ds (and dL/db) of instances whose points are split across the ranks
    of ``dist``: ``local_fn(out)`` writes this rank's partial sums into the views
    ``out = (loss, ds, db)`` (``lrnr_residual_grad`` on the rank's ``point_shard``
    with ``norm`` = the whole instances' counts), then one sum all-reduce of the
    flat buffer gives every rank the totals.  ``bufs`` (from ``partial_buffers``)
    reuses buffers across calls.  Returns the views."""
    flat, views = bufs if bufs is not None else partial_buffers(n_inst, sum_r, sum_m, want_db,
                                                               device, dtype)
    local_fn(views)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    return views


def sharded_spinprop_step(model, form: str, prec: str, shard_batch, s, m, v, step, dist,
                          bufs=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, lambda_loc=0.0,
                          s_anchor=None, loss="mse", w=None, loss_out=None):
    """One SPInProp Adam step on s for instances whose points are split across the
    ranks: the rank's residual + gradient pass (library), the all-reduce of
    (loss, dL/ds), and the replicated Adam update (library, ``lrnr_adam_update``).
    ``shard_batch`` is a ``DeviceBatch`` of the rank's points whose ``norm`` holds
    the whole instances' counts and whose coefficients are ``s``.  Returns s."""
    from . import binding as B
    if bufs is None:
        bufs = partial_buffers(shard_batch.n_inst, model.sum_r, model.sum_m, False,
                               device=s.device)
    lo, ds, _ = sharded_residual_grad(
        lambda out: B.lrnr_residual_grad(model, form, prec, shard_batch, loss=loss, w=w,
                                         want_db=False, out=out),
        shard_batch.n_inst, model.sum_r, model.sum_m, dist, want_db=False, bufs=bufs)
    B.lrnr_adam_update(ds, s, m, v, step, lr=lr, beta1=beta1, beta2=beta2, eps=eps,
                       lambda_loc=lambda_loc, s_anchor=s_anchor, loss_in=lo, loss_out=loss_out)
    return s


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank scalar (timing); identity without a process group."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
