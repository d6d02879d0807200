"""The algorithmic work model behind the benchmark's roofline figure, counted by hand
for the benchmark network (CDR, L = 5 hidden layers, M = 256, ranks (2, 16, 16, 16,
16, 1), rhat = 16 rows per layer; 65,536 interior points, 2,048 initial points and
1,024 periodic pairs)."""
import bench
import synth


def by_hand(r, rhat, C):
    # per hidden layer: reduced products y -> a (rhat x r_in) and w -> zhat (rhat x
    # r_out), forward and adjoint, 2 flops per multiply-add, C jet channels; plus 30
    # flops per row for the tanh jet and its adjoint
    tot = 0
    for l in range(len(r) - 1):
        tot += C * (2 * rhat * r[l] + 2 * rhat * r[l + 1]) * 2 + 30 * rhat
    return tot


def test_flops_per_point_of_the_benchmark_network():
    net, bt = synth.workload_cdr_single()
    assert list(net.r) == [2, 16, 16, 16, 16, 1] and net.M == 256
    rh = [16] * net.L
    assert bench.fast_flops_per_point(net.r, rh, 4) == by_hand(net.r, 16, 4) == 35_936
    assert bench.fast_flops_per_point(net.r, rh, 1) == by_hand(net.r, 16, 1) == 10_784
    n_int, n_bnd = bt.x_int.shape[0], bt.x_ic.shape[0] + 2 * bt.t_bc.shape[0]
    assert (n_int, n_bnd) == (65_536, 4_096)
    assert n_int * 35_936 + n_bnd * 10_784 == 2_399_272_960


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops x 2,070 MHz
    assert abs(bench.fp32_peak_tflops(2070.0) - 80.54784) < 1e-9


def test_clock_sampler_keeps_our_gpu_and_the_timed_region(tmp_path, monkeypatch):
    """ClockSampler against a stand-in nvidia-smi that prints two GPUs every 20 ms
    (the first lines after a 0.2 s start-up): stop() reports only the samples of the
    UUID it was given that arrived between start() and stop(), and the throttle
    reasons marked Active in them."""
    import os
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!/bin/sh\nsleep 0.2\n"
        "while true; do\n"
        "echo 'GPU-aaaa, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active'\n"
        "echo 'GPU-bbbb, 1500, 2070, 300.0, 0x0, Active, Not Active, Not Active, Not Active'\n"
        "sleep 0.02\ndone\n")
    os.chmod(fake, 0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    cs = bench.ClockSampler("GPU-AAAA")
    cs.start()
    assert cs.lines, "start() returns after the first sample"
    time.sleep(0.3)
    res = cs.stop()
    assert res["sm_mhz"] == 2070.0 and res["sm_max_mhz"] == 2070.0
    assert res["reasons"] == ["sw_power_cap"]
    assert res["samples"] >= 3
