"""Instance sharding across ranks (world size 2, gloo, CPU): each rank evaluates its
block of instances with the oracle; gathered, the blocks equal the whole batch, and
the only collective on the timing path is the max over ranks."""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import lrnr64
from paper_2410_04001_gb300 import shard


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
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


def test_instance_range_partitions():
    for n in (1, 5, 512, 1023):
        for w in (1, 2, 3, 8):
            got = [shard.instance_range(n, w, r) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [h - l for l, h in got]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_cover_the_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, ref, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    assert mx == 2.0
