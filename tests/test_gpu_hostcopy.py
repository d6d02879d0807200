"""lrnr_copy_pinned: the copy kernel between pinned host memory and the device."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    return P


def _bytes(n, seed):
    return torch.from_numpy(np.random.default_rng(seed).integers(0, 256, n, dtype=np.uint8))


@pytest.mark.parametrize("n", [1, 15, 16, 17, 255, 4096, 4099, 538_880, 1_000_003])
@pytest.mark.parametrize("soff,doff", [(0, 0), (3, 3), (5, 0), (1, 7)])
def test_copy_each_direction_bit_exact(P, n, soff, doff):
    """Host -> device, device -> host, device -> device and host -> host, at sizes with
    and without a 16-byte body and at source / destination offsets that agree or
    disagree modulo 16; the bytes around the destination range stay untouched."""
    src_h = torch.zeros(n + 32, dtype=torch.uint8).pin_memory()
    src_h[soff:soff + n] = _bytes(n, n + soff)
    src_d = src_h.cuda()
    ref = src_h[soff:soff + n].clone()
    for src, dst_dev in ((src_h, "cuda"), (src_d, "cpu"), (src_d, "cuda"), (src_h, "cpu")):
        dst = torch.full((n + 32,), 0xA5, dtype=torch.uint8, device=dst_dev)
        if dst_dev == "cpu":
            dst = dst.pin_memory()
        P.lrnr_copy_pinned(dst[doff:doff + n], src[soff:soff + n])
        torch.cuda.synchronize()
        out = dst.cpu()
        assert torch.equal(out[doff:doff + n], ref)
        assert torch.all(out[:doff] == 0xA5) and torch.all(out[doff + n:] == 0xA5)


def test_copy_typed_views_and_empty(P):
    x = torch.randn(3, 1000).pin_memory()
    y = torch.empty(3, 1000, device="cuda")
    P.lrnr_copy_pinned(y, x)
    z = torch.empty(3, 1000).pin_memory()
    P.lrnr_copy_pinned(z, y)
    torch.cuda.synchronize()
    assert torch.equal(z, x)
    e = torch.empty(0, device="cuda")
    P.lrnr_copy_pinned(e, torch.empty(0).pin_memory())     # no launch, no error


def test_captured_copy_reads_host_writes_between_replays(P):
    """A graph holding host -> device, a device kernel and device -> host: each replay
    sees the values the host wrote into the pinned source since the previous one."""
    n = 100_000
    h_in = torch.zeros(n).pin_memory()
    h_out = torch.zeros(n).pin_memory()
    d = torch.zeros(n, device="cuda")
    d2 = torch.zeros(n, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        P.lrnr_copy_pinned(d, h_in)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        P.lrnr_copy_pinned(d, h_in)
        torch.mul(d, 2.0, out=d2)
        P.lrnr_copy_pinned(h_out, d2)
    for k in range(4):
        h_in.copy_(torch.arange(n, dtype=torch.float32) * (k + 1))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(h_out, torch.arange(n, dtype=torch.float32) * (2 * (k + 1)))


def test_copy_rejects_pageable_overlap_and_null(P):
    from paper_2410_04001_gb300 import binding as B
    lib = B.lib()
    pageable = np.zeros(64, dtype=np.uint8)
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    hp = ctypes.c_void_p(pageable.ctypes.data)
    dp = ctypes.c_void_p(d.data_ptr())
    assert lib.lrnr_copy_pinned(dp, hp, 64, st) == B.EINVAL
    assert lib.lrnr_copy_pinned(hp, dp, 64, st) == B.EINVAL
    assert lib.lrnr_copy_pinned(None, dp, 64, st) == B.EINVAL
    assert lib.lrnr_copy_pinned(ctypes.c_void_p(d.data_ptr() + 8), dp, 32, st) == B.EINVAL
    assert lib.lrnr_copy_pinned(None, None, 0, st) == B.OK
    with pytest.raises(ValueError):
        P.lrnr_copy_pinned(d, torch.zeros(64, dtype=torch.uint8))          # CPU, not pinned
    with pytest.raises(ValueError):
        P.lrnr_copy_pinned(d, torch.zeros(65, dtype=torch.uint8).pin_memory())
    torch.cuda.synchronize()
