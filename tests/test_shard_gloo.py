"""Data-parallel splits on CPU ranks (gloo, world size 2).

Instance sharding: each rank evaluates its block of instances with the oracle;
gathered, the blocks equal the whole batch, and the only collective on the timing
path is the max over ranks.

Point sharding within an instance (the loss of Eq. 3.5 is a sum over points over
the point counts, so the gradient is a sum over points, Sec. 2.3): each rank takes
its block of every instance's points (``shard.point_shard``), evaluates them with
the oracle using the whole instances' counts, and ``shard.sharded_residual_grad``
all-reduces (loss, dL/ds, dL/db) once; the result equals the unsharded oracle to
1e-12.  (The CUDA library cannot run on CPU ranks: the oracle stands in for the
per-rank evaluation, the split and the collective are the product's.)"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import lrnr64
from paper_2410_04001_gb300 import shard


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _instance_worker(rank, world, port, q):
    _init(rank, world, port)
    try:
        g = synth.rng(5)
        net = synth.make_net(g, L=2, M=12, r=4)
        bt = synth.make_instances(g, net, 5, 20, 60)
        lo, hi = shard.instance_range(bt.n_inst, world, rank)
        part = shard.subset(bt, lo, hi)
        losses, ds, _ = lrnr64.residual_grad(net, part, "full")
        t = torch.zeros(bt.n_inst, dtype=torch.float64)
        t[lo:hi] = torch.tensor(losses)
        dist.all_reduce(t)            # gather for the check only
        mx = shard.max_over_ranks(float(rank + 1), dist)
        if rank == 0:
            ref, _, _ = lrnr64.residual_grad(net, bt, "full")
            q.put((t.numpy().tolist(), ref.tolist(), mx))
    finally:
        dist.destroy_process_group()


def _ragged_case():
    g = synth.rng(11)
    net = synth.make_net(g, L=2, M=16, r=4)
    # instance 1 has a single interior point (one rank gets none), instance 2 no
    # initial points, instance 3 an odd number of pairs
    bt = synth.make_batch(g, net, [41, 1, 30, 17], [7, 4, 0, 5], [5, 2, 3, 9],
                          [5.0, 2.0, 9.0, 1.5], [1.0, 0.0, 2.0, 0.3], [2.0, 1.0, 0.0, 4.0])
    return net, bt


def _point_worker(rank, world, port, q):
    _init(rank, world, port)
    try:
        net, bt = _ragged_case()
        part, counts = shard.point_shard(bt, world, rank)
        res = {}
        for loss in ("mse", "l1"):
            def local(out, loss=loss):
                lo, ds, db = lrnr64.residual_grad(net, part, "full", loss=loss, counts=counts)
                out[0].copy_(torch.from_numpy(lo))
                out[1].copy_(torch.from_numpy(ds))
                out[2].copy_(torch.from_numpy(db))
            views = shard.sharded_residual_grad(local, bt.n_inst, net.sum_r, net.sum_m, dist,
                                                want_db=True, dtype=torch.float64)
            res[loss] = [v.numpy().copy() for v in views]
        if rank == 0:
            q.put(res)
    finally:
        dist.destroy_process_group()


def _run(target, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000) + (0 if target is _instance_worker else 1)
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


def test_instance_range_partitions():
    for n in (0, 1, 5, 512, 1023):
        for w in (1, 2, 3, 8):
            got = [shard.instance_range(n, w, r) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [h - l for l, h in got]
            assert max(sizes) - min(sizes) <= 1


def test_point_shards_cover_every_point_once():
    _, bt = _ragged_case()
    for world in (1, 2, 3, 5):
        parts = [shard.point_shard(bt, world, r) for r in range(world)]
        for _, counts in parts:
            assert np.array_equal(counts, shard.instance_counts(bt))
        for i in range(bt.n_inst):
            ref = bt.instance(i)
            got = [p.instance(i) for p, _ in parts]
            for k in ("x_int", "t_int", "x_ic", "t_bc"):
                assert np.array_equal(np.concatenate([g_[k] for g_ in got]), ref[k]), (world, i, k)


@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_oracle_shards_with_whole_counts_add_up_to_the_instance(loss):
    """The count override of the oracle pinned against its own unsharded path: the
    per-point terms of every shard, each divided by the whole instance's counts,
    sum to the instance's loss and gradient."""
    net, bt = _ragged_case()
    ref = lrnr64.residual_grad(net, bt, "full", loss=loss)
    for world in (2, 3):
        tot = [0.0, 0.0, 0.0]
        for r in range(world):
            part, counts = shard.point_shard(bt, world, r)
            out = lrnr64.residual_grad(net, part, "full", loss=loss, counts=counts)
            tot = [a + b for a, b in zip(tot, out)]
        for a, b in zip(tot, ref):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-15)


def test_two_gloo_ranks_cover_the_batch():
    got, ref, mx = _run(_instance_worker)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    assert mx == 2.0


def test_two_gloo_ranks_point_sharded_gradient_equals_unsharded():
    res = _run(_point_worker)
    net, bt = _ragged_case()
    for loss in ("mse", "l1"):
        ref = lrnr64.residual_grad(net, bt, "full", loss=loss)
        for a, b in zip(res[loss], ref):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-15), loss
