"""Benchmark of the FastLRNR / SPInProp hot path on one GB300 (or N replicas).

Workload: the single-instance convection-diffusion-reaction problem
(beta = 5, nu = 1, rho = 2) on an LRNR with L = 5 hidden layers of width M = 256
and rank r = 16, FastLRNR with 16 EIM rows per layer; 65,536 interior points,
2,048 initial points and 1,024 periodic pairs (69,632 collocation points).

A step is one fused SPInProp pass through the C ABI (``spinprop_step``, one Adam
step): input jets, reduced layers, output, CDR residual, loss and seeds, adjoint
sweep, fixed-order gradient reduction and the Adam update of s.  The metric is
collocation points per second.  The same run times the full-width FP32 LRNR
residual + gradient on the same batch (``variants``) and measures the error of
each path against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "residual+grad points/s, FastLRNR & full LRNR, BF16 vs FP32, err vs FP64 oracle"
WORKLOAD = ("CDR beta=5 nu=1 rho=2; LRNR L=5 hidden layers, M=256, r=16, tanh; FastLRNR "
            "rhat=16 rows/layer (EIM); 65,536 interior + 2,048 initial + 1,024 periodic pairs")


def workload_name(world):
    """One instance of the CDR problem with world x (65,536 + 2,048 + 1,024 pairs)
    points; on N ranks each rank takes its block of every point class."""
    if world == 1:
        return WORKLOAD
    return (WORKLOAD.replace("65,536 interior + 2,048 initial + 1,024 periodic pairs",
                             f"{world} x (65,536 interior + 2,048 initial + 1,024 periodic pairs)")
            + f", points split over {world} ranks")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error and CPU baseline")
    ap.add_argument("--no-configs", action="store_true", help="skip the batched / SPInProp workloads")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="collective backend at N ranks (gloo: host-side all-reduce)")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one kernel case --steps times (for profilers) and exit")
    return ap.parse_args()


# --------------------------------------------------------------------------- profiling cases

PROFILE_CASES = {
    "fast_fp32_cdr": "FastLRNR SPInProp step, FP32 (k_fast + reduction / Adam), CDR M=256 r=16 L=5, 69,632 points",
    "fastk_fp32_paper_d2": "FastLRNR SPInProp step, FP32 reduced coordinates (k_fastk), M=4000 r=(1,49,30,25,1) "
                           "rhat=5, 65,536 + 2,048 + 1,024 pairs",
    "fast_bf16_cdr": "FastLRNR SPInProp step, reduced network on BF16 tensor cores (k_full_tc), CDR M=256 "
                     "r=16 L=5, 69,632 points",
    "fast_tf32_cdr": "FastLRNR SPInProp step, reduced network on TF32 tensor cores (k_full_tc), CDR M=256 "
                     "r=16 L=5, 69,632 points",
    "full_bf16_cdr": "full-width residual + gradient, BF16 tensor cores (k_full_tc), CDR M=256 r=16 L=5",
    "full_tf32_cdr": "full-width residual + gradient, TF32 tensor cores (k_full_tc), CDR M=256 r=16 L=5",
    "full_bf16x3_cdr": "full-width residual + gradient, split-BF16 tensor cores (k_full_tc), CDR M=256 r=16 L=5",
    "full_fp32_cdr": "full-width residual + gradient, FP32 SIMT (k_full_fp32), CDR M=256 r=16 L=5",
    "full_fp32_stress": "full-width residual + gradient, FP32 SIMT at rank 32 (k_full_fp32_sl, two threads "
                        "per point), M=1024 r=32 L=6, 262,144 points",
    "full_fp32_paper_d2": "full-width SPInProp step, FP32 SIMT at rank 64 (k_full_fp32_sl, four threads per "
                          "point), M=4000 r=(1,49,30,25,1), 65,536 + 2,048 + 1,024 pairs",
}


def run_profile_case(args):
    """Build the case's model and batch, run it --warmup + --steps times on the
    current stream, print one line with the mean CUDA-event time per call."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    import synth
    from paper_2410_04001_gb300 import fastphase
    dev = torch.device("cuda", 0)
    case = args.profile_case
    if case in ("fastk_fp32_paper_d2", "full_fp32_paper_d2"):
        net, bx, bt = synth.workload_paper_d2()
    elif case == "full_fp32_stress":
        net, bt = synth.workload_adjoint_stress()
    else:
        net, bt = synth.workload_cdr_single()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt, dev)
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    if case.startswith("fast"):
        s0 = bt.s[:1]
        fastphase.build_reduced(model, torch.tensor(xs, device=dev), torch.tensor(ts, device=dev),
                                torch.tensor(s0, device=dev), rhat=5 if case.startswith("fastk") else 16)
        s = db.s.clone()
        m, v = torch.zeros_like(s), torch.zeros_like(s)
        k = torch.zeros(1, dtype=torch.int64, device=dev)
        fprec = case.split("_")[1]
        fn = lambda: P.spinprop_step(model, "fast", fprec, db, s, m, v, k, 1, lr=1e-3)
    elif case == "full_fp32_paper_d2":
        s = db.s.clone()
        m, v = torch.zeros_like(s), torch.zeros_like(s)
        k = torch.zeros(1, dtype=torch.int64, device=dev)
        fn = lambda: P.spinprop_step(model, "full", "fp32", db, s, m, v, k, 1, lr=1e-3)
    else:
        prec = case.split("_")[1]
        out = P.lrnr_residual_grad(model, "full", prec, db, want_db=False)
        fn = lambda: P.lrnr_residual_grad(model, "full", prec, db, out=out, want_db=False)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "what": PROFILE_CASES[case], "points": db.n_points,
                      "calls": args.steps, "ms_per_call": e0.elapsed_time(e1) / max(1, args.steps),
                      "device_status": P.lrnr_last_device_status(model)}))


# --------------------------------------------------------------------------- peaks

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes (read + write) per launch of the FastLRNR kernel on this workload, from
# one ncu capture of the current kernel (the mean of three launches of
# dram__bytes_read.sum + dram__bytes_write.sum), or None while the kernel has
# changed since the last capture.
K_FAST_DRAM_BYTES = 50_856_874

GB300_SMS = 152
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return GB300_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# --------------------------------------------------------------------------- flops model

def fast_flops_per_point(r, rhat, channels):
    """Algorithmic FP32 flops of one point through the FastLRNR forward + adjoint
    (no recomputation counted): per hidden layer 2*C*rh*(2*r_in + 2*r_out) for the
    four reduced products, plus ~30 flops per row for the tanh jet and its adjoint."""
    L = len(r) - 1
    tot = 0
    for l in range(L):
        tot += 2 * channels * rhat[l] * (2 * r[l] + 2 * r[l + 1]) + 30 * rhat[l]
    return tot


def full_flops_per_point(r, M, channels):
    L = len(r) - 1
    tot = 0
    for l in range(L):
        tot += 2 * channels * M * (2 * r[l] + 2 * r[l + 1]) + 30 * M
    return tot


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while the timed region
    runs.  Every GPU nvidia-smi lists is sampled (no --id: its id forms differ between
    driver versions); stop() keeps the lines of the GPU whose UUID torch reports, or
    all lines when nvidia-smi lists a single GPU.  start() returns once the first
    sample has arrived (nvidia-smi takes a while to start), and stop() keeps the
    samples that arrived between the two calls (the latest earlier ones if none did)."""
    QUERY = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = (uuid or "").lower().replace("gpu-", "")
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t_end = time.perf_counter() + 10.0
            while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t_start = time.perf_counter()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t_stop = time.perf_counter()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for ts, ln in self.lines if self.t_start <= ts <= t_stop]
        if not inside:
            inside = [ln for ts, ln in self.lines if ts < self.t_start][-8:]   # one line per GPU
        rows = [[x.strip() for x in ln.split(",")] for ln in inside]
        rows = [f for f in rows if len(f) >= 9]
        uuids = {f[0].lower().replace("gpu-", "") for f in rows}
        if self.uuid in uuids:
            rows = [f for f in rows if f[0].lower().replace("gpu-", "") == self.uuid]
        elif len(uuids) > 1:
            rows = []          # several GPUs and none is ours: report no samples
        for f in rows:
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU baseline

def cpu_baseline_child():
    """Runs in a fresh interpreter: time the FP64 oracle's SPInProp step (FastLRNR
    residual + gradient + Adam) on a bounded sample of the workload."""
    import numpy as np
    import synth
    from oracle import adam64, eim64, lrnr64
    net, bt = synth.workload_cdr_single()
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _ = eim64.eim_greedy(lrnr64.hidden_states(net, bt.s[0], xs, ts, l), 16)
        rows.append(p)
        Xis.append(Xi)
    fnet = lrnr64.make_fast(net, rows, Xis)
    inst = bt.instance(0)
    s = inst["s"].copy()
    m = np.zeros_like(s)
    v = np.zeros_like(s)
    n_pts = bt.n_points
    t0 = time.perf_counter()
    k = 0
    while True:
        k += 1
        _, gs, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet,
                                             dict(inst, s=s))
        s, m, v = adam64.adam_step(s, m, v, k, gs)
        if time.perf_counter() - t0 > float(os.environ.get("LRNR_CPU_SECONDS", "12")) or k >= 50:
            break
    dt = time.perf_counter() - t0
    print(json.dumps({"value": n_pts * k / dt, "steps": k, "seconds": dt, "points": n_pts}))


def _cpu_child(threads, seconds):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    env["LRNR_CPU_SECONDS"] = str(seconds)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-child"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return (json.loads(line[-1]), None) if line else (None, r.stderr[-300:])


def run_cpu_baseline():
    """The oracle's step on the host cores: all of them (the reported value) and one
    BLAS thread (reported beside it)."""
    cores = len(os.sched_getaffinity(0))
    d, err = _cpu_child(cores, 12)
    if d is None:
        return {"value": None, "unit": "points/s", "cores": cores, "kind": "oracle",
                "sample": "failed: " + err}
    d1, _ = _cpu_child(1, 6)
    return {"value": d["value"], "unit": "points/s", "cores": cores, "kind": "oracle",
            "value_1_thread": d1["value"] if d1 else None,
            "sample": (f"FP64 NumPy oracle, FastLRNR SPInProp step (residual + gradient + Adam) "
                       f"over the full 69,632-point batch, {d['steps']} steps in {d['seconds']:.1f} s; "
                       f"BLAS threads = {cores} (value_1_thread: the same with one BLAS thread, "
                       f"{d1['steps'] if d1 else 0} steps).  The oracle's step is a chain of small "
                       f"NumPy operations, not BLAS-bound: it runs on one core in effect, and the "
                       f"extra BLAS threads do not speed it up")}


# --------------------------------------------------------------------------- reference arm

def run_reference(args):
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    import numpy as np
    import synth
    from oracle import adam64, eim64, lrnr64
    net, bt = synth.workload_cdr_single(scale=world)
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _ = eim64.eim_greedy(lrnr64.hidden_states(net, bt.s[0], xs, ts, l), 16)
        rows.append(p)
        Xis.append(Xi)
    fnet = lrnr64.make_fast(net, rows, Xis)
    inst = bt.instance(0)

    def sample(stride):
        d = dict(inst)
        d["x_int"], d["t_int"] = inst["x_int"][::stride], inst["t_int"][::stride]
        d["x_ic"], d["t_bc"] = inst["x_ic"][::stride], inst["t_bc"][::stride]
        return d, len(d["x_int"]) + len(d["x_ic"]) + 2 * len(d["t_bc"])

    # each step: the oracle SPInProp step on a bounded sample (every stride-th point
    # of each class), the stride chosen so that warm-up + K steps take about 90 s
    cal, ncal = sample(8)
    t0 = time.perf_counter()
    lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet, cal)
    per_point = (time.perf_counter() - t0) / ncal
    budget = 90.0 / max(1, args.steps + args.warmup)
    stride = max(1, int(np.ceil(bt.n_points * per_point / budget)))
    sub, n_pts = sample(stride)
    s = inst["s"].copy()
    m = np.zeros_like(s)
    v = np.zeros_like(s)
    k = 0

    def step():
        nonlocal s, m, v, k
        k += 1
        _, gs, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet, dict(sub, s=s))
        s, m, v = adam64.adam_step(s, m, v, k, gs)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = n_pts * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(world) + f"; FastLRNR SPInProp step on a 1/{stride} point sample",
                   "form": "fast"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"every {stride}th point of each class ({n_pts} points per step)"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))



# --------------------------------------------------------------------------- other workloads

def select_rows_on_device(P, model, net, s0, dev, torch, synth):
    """Device snapshots at the 4 x 3 design plus perturbations, device EIM; returns the
    rows the device selected per layer."""
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    xs_d, ts_d = torch.tensor(xs, device=dev), torch.tensor(ts, device=dev)
    rows = []
    for l in range(net.L):
        S = P.lrnr_snapshots(model, l, xs_d, ts_d, torch.tensor(s0[None, :], device=dev))
        r, _, _ = P.fastlrnr_select_rows(model, l, S, 16)
        rows.append(r.cpu().numpy())
    return rows


def oracle_fast_net(P, model, net, s0, synth, torch, dev):
    """The oracle's own FastLRNR for the same construction (its exact-LRNR snapshots at
    the same design, its greedy EIM), installed on the device model as well, so that
    the kernels' errors are measured on one reduced network.  (The device's own
    selection, from its own snapshots, can differ at the deep layers, whose snapshot
    spectra fall below rounding after about ten modes.)  Returns the oracle network
    and its rows."""
    from oracle import eim64, lrnr64
    xs, ts = synth.snapshot_design(synth.rng(77), 8)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _ = eim64.eim_greedy(lrnr64.hidden_states(net, s0, xs, ts, l), 16)
        rows.append(p)
        Xis.append(Xi)
        P.fastlrnr_select_rows(model, l, None, len(p),
                               rows_in=torch.tensor(p.astype("int32"), device=dev),
                               Xi_in=torch.tensor(Xi.T.copy(), device=dev))
    return lrnr64.make_fast(net, rows, Xis), rows


def config_variants(P, synth, np, torch, dev, timed_steps, peak, with_oracle):
    """Batched CDR instances (512, log-uniform counts) and the 1,024-instance SPInProp
    loop, FastLRNR FP32; plus the fast-phase loop against the same loop on the
    full-width FP32 LRNR (200 Adam steps on 16 instances)."""
    out = {}
    # 512 instances, ~7.9 M points, one residual + gradient pass: the tile shape picked
    # by the autotuner, the call replayed from a captured CUDA graph
    from paper_2410_04001_gb300.autotune import autotune
    net, bt = synth.workload_batched()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    rows_dev = select_rows_on_device(P, model, net, bt.s[0], dev, torch, synth)
    db = P.DeviceBatch.from_host(bt, dev)
    tuned = autotune(model, db, "fast", "fp32", cache=None, reps=3)
    res = P.lrnr_residual_grad(model, "fast", "fp32", db)
    P.lrnr_timing(model, True)
    _, km, kn = timed_steps(lambda: P.lrnr_residual_grad(model, "fast", "fp32", db, out=res), 5, model)
    P.lrnr_timing(model, False)
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, capture_error_mode="relaxed"):
        P.lrnr_residual_grad(model, "fast", "fp32", db, out=res)
    gr.replay()
    ts_, _, _ = timed_steps(gr.replay, 10)
    ms = sum(ts_) / len(ts_)
    r = {"workload": "512 CDR instances, counts log-uniform [1,024, 65,536], M=256 r=16 L=5 rhat=16",
         "points": db.n_points, "points_per_s": db.n_points / (ms * 1e-3), "ms_per_call": ms,
         "kernel_ms": km / max(1, kn), "cuda_graph": True,
         "autotuned_shape": {"nt": tuned["nt"], "ctas_per_sm": tuned["ctas_per_sm"]}}
    if with_oracle:
        from oracle import lrnr64
        fnet, rows_o = oracle_fast_net(P, model, net, bt.s[0], synth, torch, dev)
        r["eim_rows_match_oracle"] = all(np.array_equal(a, b) for a, b in zip(rows_o, rows_dev))
        res = P.lrnr_residual_grad(model, "fast", "fp32", db)
        f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        errs = []
        for i in (0, 255, 511):
            inst = bt.instance(i)
            inst = {k: (f32(v) if isinstance(v, np.ndarray) else float(np.float32(v))) for k, v in inst.items()}
            ro, rs, _ = lrnr64.instance_loss_grad(lrnr64.fast_forward, lrnr64.fast_backward, fnet, inst)
            ds = res[1][i].cpu().numpy()
            errs.append(float(np.linalg.norm(ds - rs) / np.linalg.norm(rs)))
        r["err_dL_ds_sampled_instances"] = max(errs)
    out["batched_512_fast_fp32"] = r
    # the same batch through the reduced network on the tensor cores (BF16)
    res16 = P.lrnr_residual_grad(model, "fast", "bf16", db)
    P.lrnr_timing(model, True)
    ts_, km, kn = timed_steps(lambda: P.lrnr_residual_grad(model, "fast", "bf16", db, out=res16), 10, model)
    P.lrnr_timing(model, False)
    ms = sum(ts_) / len(ts_)
    ds32, ds16 = res[1].double(), res16[1].double()
    out["batched_512_fast_bf16"] = {
        "workload": r["workload"], "points": db.n_points, "points_per_s": db.n_points / (ms * 1e-3),
        "ms_per_call": ms, "kernel_ms": km / max(1, kn),
        "dL_ds_rel_diff_vs_fp32": float((ds16 - ds32).norm() / ds32.norm())}
    del model, db, res, res16
    # 1,024 instances x 16,384 points, fused SPInProp steps
    net, bt = synth.workload_spinprop()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    select_rows_on_device(P, model, net, bt.s[0], dev, torch, synth)
    db = P.DeviceBatch.from_host(bt, dev)
    s = db.s.clone()
    m, v = torch.zeros_like(s), torch.zeros_like(s)
    k = torch.zeros(1, dtype=torch.int64, device=dev)
    P.spinprop_step(model, "fast", "fp32", db, s, m, v, k, 2)
    ts_, _, _ = timed_steps(lambda: P.spinprop_step(model, "fast", "fp32", db, s, m, v, k, 1), 10)
    ms = sum(ts_) / len(ts_)
    s16, m16, v16 = db.s.clone(), torch.zeros_like(s), torch.zeros_like(s)
    k16 = torch.zeros(1, dtype=torch.int64, device=dev)
    P.spinprop_step(model, "fast", "bf16", db, s16, m16, v16, k16, 2)
    ts16, _, _ = timed_steps(lambda: P.spinprop_step(model, "fast", "bf16", db, s16, m16, v16, k16, 1), 10)
    ms16 = sum(ts16) / len(ts16)
    out["spinprop_1024_fast_bf16"] = {"points": db.n_points, "steps_per_s": 1e3 / ms16,
                                      "points_per_s": db.n_points / (ms16 * 1e-3), "ms_per_step": ms16}
    out["spinprop_1024_fast_fp32"] = {
        "workload": "1,024 CDR instances x 16,384 points, M=512 r=16 L=5 rhat=16, one Adam step",
        "points": db.n_points, "steps_per_s": 1e3 / ms, "points_per_s": db.n_points / (ms * 1e-3),
        "ms_per_step": ms}
    # fast phase vs full-width fine-tune: 200 Adam steps on the first 16 instances
    from paper_2410_04001_gb300 import shard
    sub = shard.subset(bt, 0, 16)
    dsub = P.DeviceBatch.from_host(sub, dev)
    cmp = {}
    for form in ("fast", "full"):
        s = dsub.s.clone()
        m, v = torch.zeros_like(s), torch.zeros_like(s)
        k = torch.zeros(1, dtype=torch.int64, device=dev)
        lo = torch.zeros(16, dtype=torch.float32, device=dev)
        P.spinprop_step(model, form, "fp32", dsub, s, m, v, k, 1, loss_out=lo)
        torch.cuda.synchronize()
        l0 = float(lo.mean())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.spinprop_step(model, form, "fp32", dsub, s, m, v, k, 199, loss_out=lo)
        e1.record()
        torch.cuda.synchronize()
        # residual loss of the final s, always measured on the full-width LRNR
        lf, _, _ = P.lrnr_residual_grad(model, "full", "fp32", dsub.with_s(s), want_db=False)
        cmp[form] = {"steps_per_s": 199e3 / e0.elapsed_time(e1), "loss_first_step": l0,
                     "final_full_lrnr_loss": float(lf.mean())}
    out["spinprop_fast_vs_full_16_instances"] = cmp
    del model, db, dsub
    out["paper_d1_fast_phase"] = paper_fast_phase(P, synth, np, torch, dev)
    out["paper_d2_fast_phase"] = paper_fast_phase(P, synth, np, torch, dev, d2=True)
    out["eim_vs_deim_rhat_sweep"] = eim_vs_deim(P, synth, np, torch, dev)
    out.update(small_and_stress(P, synth, np, torch, dev, timed_steps, with_oracle))
    return out


def small_and_stress(P, synth, np, torch, dev, timed_steps, with_oracle):
    """The latency case (M = 64, r = 8, L = 4, pure convection, 1,408 points: microseconds
    per residual + gradient call, FP32 full width and FastLRNR) and the full-width
    adjoint stress case (M = 1,024, r = 32, L = 6, 262,144 points: FP32, BF16, TF32
    and split-BF16), each a residual + gradient call with the L2 flushed before it; dL/ds
    of the stress case against the oracle on a 1,024-point sub-batch."""
    out = {}
    net, bt = synth.workload_convection_small()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    select_rows_on_device(P, model, net, bt.s[0], dev, torch, synth)
    db = P.DeviceBatch.from_host(bt, dev)
    r = {"workload": "M=64 r=8 L=4 convection beta=5; 1,024 + 256 + 128 pairs", "points": db.n_points}
    for form in ("full", "fast"):
        res = P.lrnr_residual_grad(model, form, "fp32", db)
        ts_, _, _ = timed_steps(lambda: P.lrnr_residual_grad(model, form, "fp32", db, out=res), 50)
        r[form + "_fp32_us_per_call"] = 1e3 * sum(ts_) / len(ts_)
    out["latency_small_convection"] = r
    del model, db
    net, bt = synth.workload_adjoint_stress()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    db = P.DeviceBatch.from_host(bt, dev)
    n = db.n_points
    r = {"workload": "M=1024 r=32 L=6 CDR; 262,144 interior points, full width", "points": n}
    if with_oracle:
        from oracle import lrnr64
        f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        sub = synth.Batch(beta=f32(bt.beta), nu=f32(bt.nu), rho=f32(bt.rho), s=f32(bt.s),
                          int_off=np.array([0, 1024]), ic_off=np.array([0, 0]), bc_off=np.array([0, 0]),
                          x_int=f32(bt.x_int[:1024]), t_int=f32(bt.t_int[:1024]), x_ic=np.zeros(0),
                          t_bc=np.zeros(0))
        _, rs, _ = lrnr64.residual_grad(net, sub, "full")
        dsub = P.DeviceBatch.from_host(sub, dev)
    for prec in ("fp32", "bf16", "tf32", "bf16x3"):
        res = P.lrnr_residual_grad(model, "full", prec, db, want_db=False)
        P.lrnr_timing(model, True)
        ts_, km, kn = timed_steps(lambda: P.lrnr_residual_grad(model, "full", prec, db, out=res,
                                                               want_db=False), 3, model)
        P.lrnr_timing(model, False)
        ms = sum(ts_) / len(ts_)
        e = {"ms_per_call": ms, "kernel_ms": km / max(1, kn), "points_per_s": n / (ms * 1e-3)}
        if with_oracle:
            _, ds, _ = P.lrnr_residual_grad(model, "full", prec, dsub, want_db=False)
            e["err_dL_ds_1024_points"] = float(np.linalg.norm(ds.cpu().numpy() - rs) / np.linalg.norm(rs))
        r[prec] = e
    out["full_width_adjoint_stress"] = r
    del model, db
    return out


def eim_vs_deim(P, synth, np, torch, dev):
    """Accuracy of the reduced network against the full one as a function of rhat,
    for the two ways of choosing (Xi, P) in Eq. 2.7: greedy EIM on the snapshots and
    POD + DEIM.  Metric: mean absolute difference u_FAST - u_LRNR over a uniform
    256 x 64 grid of the domain (the measure of Fig. 2), at the coefficients the
    snapshots were taken around (s0) and at s0 perturbed by 5 % (unseen); FP32
    kernels, snapshots from 8 coefficient draws around s0 at the 4 x 3 design plus
    8 perturbations per point."""
    xg, tg = np.meshgrid(np.linspace(0, 2 * np.pi, 256), np.linspace(0, 1, 64), indexing="ij")
    out = {}
    cases = (("cdr_M256_r16_L5", synth.workload_cdr_single()[0], 1005),
             ("paper_d1_M4000_r(1,5,5,3,1)", synth.workload_paper_d1()[0], 1006))
    for name, net, seed in cases:
        g = synth.rng(seed)
        model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
        s0 = synth.make_s(g, 1, sum(net.r))[0]
        draws = np.stack([s0] + [s0 * (1.0 + 0.1 * g.standard_normal(s0.shape)) for _ in range(7)])
        s1 = s0 * (1.0 + 0.05 * g.standard_normal(s0.shape))
        xs, ts = synth.snapshot_design(synth.rng(77), 8)
        xs_d, ts_d = torch.tensor(xs, device=dev), torch.tensor(ts, device=dev)
        S = [P.lrnr_snapshots(model, l, xs_d, ts_d, torch.tensor(draws, device=dev))
             for l in range(net.L)]
        grid = lambda s: P.DeviceBatch.from_host(synth.Batch(
            beta=np.array([1.0]), nu=np.array([0.0]), rho=np.array([0.0]), s=s[None, :],
            int_off=np.array([0, xg.size]), ic_off=np.array([0, 0]), bc_off=np.array([0, 0]),
            x_int=xg.ravel(), t_int=tg.ravel(), x_ic=np.zeros(0), t_bc=np.zeros(0)), dev)
        batches = {"s0": grid(s0), "s0_perturbed_5pct": grid(s1)}
        ref = {k: P.lrnr_residual(model, "full", "fp32", b)["u"].double() for k, b in batches.items()}
        rows = []
        for rh in (2, 4, 6, 8, 12, 16):
            row = {"rhat": rh}
            for method in ("eim", "deim"):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for l in range(net.L):
                    if method == "eim":
                        P.fastlrnr_select_rows(model, l, S[l], rh)
                    else:
                        P.fastlrnr_select_rows_deim(model, l, S[l], rh, n_iter=20)
                e1.record()
                torch.cuda.synchronize()
                row[method + "_select_ms"] = e0.elapsed_time(e1)
                for k, b in batches.items():
                    uf = P.lrnr_residual(model, "fast", "fp32", b)["u"].double()
                    row[f"{method}_mae_{k}"] = float((uf - ref[k]).abs().mean())
            rows.append(row)
        out[name] = {"mean_abs_u_LRNR_s0": float(ref["s0"].abs().mean()), "sweep": rows}
        del model
    return out


def paper_fast_phase(P, synth, np, torch, dev, d2=False):
    """The fast phase on the paper's convection architecture in shape (M = 4,000,
    r = (1, 5, 5, 3, 1), rhat = 5, X = 12 points, l1 loss + locality, Adam), against a
    full-width fine-tune Adam step (MSE over 69,632 collocation points), both FP32
    and graph-captured; the paper quotes 0.004 s vs 0.14 s per step on a V100 for its
    rank-49 architecture (context only)."""
    from paper_2410_04001_gb300 import fastphase
    net, bx, bt = synth.workload_paper_d2() if d2 else synth.workload_paper_d1()
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    s0 = bx.s[0]
    draws = np.stack([s0] + [s0 * (1.0 + 0.1 * g.standard_normal(s0.shape)) for _ in range(7)])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fastphase.build_reduced(model, torch.tensor(xs, device=dev), torch.tensor(ts, device=dev),
                            torch.tensor(draws, device=dev), rhat=5)
    e1.record()
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    dX = P.DeviceBatch.from_host(bx, dev)
    dT = P.DeviceBatch.from_host(bt, dev)
    res = {"workload": ("M=4000, r=(1,49,30,25,1), CDR mu=(2,1,1); fast phase in FP32 on the "
                        "reduced-coordinate kernel (rank 49 pads to 64), fine-tune in FP32 (four "
                        "threads per point) and in BF16 on the tensor cores" if d2 else
                        "M=4000, r=(1,5,5,3,1), convection beta=7") +
                       "; fast phase on the 12-point 4x3 grid (l1 + locality 1e-3, lr 1e-3); "
                       "fine-tune on 65,536 + 2,048 + 1,024 pairs (MSE)", "build_reduced_ms": build_ms}
    fprec = "fp32"

    def step_time(form, batch, loss, lam, reps=200, prec="fp32"):
        s = batch.s.clone()
        anchor = s.clone()
        m, v = torch.zeros_like(s), torch.zeros_like(s)
        k = torch.zeros(1, dtype=torch.int64, device=dev)
        lo = torch.zeros(1, dtype=torch.float32, device=dev)
        fn = lambda: P.spinprop_step(model, form, prec, batch, s, m, v, k, 1, lr=1e-3,
                                     lambda_loc=lam, s_anchor=anchor, loss=loss, loss_out=lo)
        for _ in range(3):
            fn()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, capture_error_mode="relaxed"):
            fn()
        for _ in range(3):
            gr.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            gr.replay()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e3 / reps

    fast_us = step_time("fast", dX, "l1", 1e-3, prec=fprec)
    fast_bf16_us = step_time("fast", dX, "l1", 1e-3, prec="bf16")
    # the reduced network on the fine-tune batch: throughput rather than latency
    big = {prec: step_time("fast", dT, "mse", 0.0, reps=50, prec=prec) for prec in ("fp32", "bf16")}
    n_big = dT.n_points
    full_us = step_time("full", dT, "mse", 0.0, reps=5 if d2 else 20)
    full_bf16_us = step_time("full", dT, "mse", 0.0, reps=20, prec="bf16")
    # the whole fast phase: 400 Adam steps (the paper's epoch budget) in one call
    e0.record()
    s_fast = fastphase.fast_phase(model, dX, 400, lr=1e-3, lambda_loc=1e-3, prec=fprec)
    e1.record()
    torch.cuda.synchronize()
    lprec = "fp32"
    lf0, _, _ = P.lrnr_residual_grad(model, "full", lprec, dT, want_db=False)
    lf1, _, _ = P.lrnr_residual_grad(model, "full", lprec, dT.with_s(s_fast), want_db=False)
    res.update({"fast_step_us": fast_us, "fast_prec": fprec, "fast_step_bf16_us": fast_bf16_us,
                "finetune_loss_prec": lprec, "full_finetune_step_us": full_us,
                "fast_step_on_finetune_batch_us": big,
                "fast_points_per_s_on_finetune_batch": {k: n_big / (v * 1e-6)
                                                        for k, v in big.items()},
                "full_finetune_step_bf16_us": full_bf16_us,
                "full_bf16_over_fast_step_ratio": full_bf16_us / fast_us,
                "full_fp32_over_fast_step_ratio": full_us / fast_us,
                "fast_phase_400_steps_ms": e0.elapsed_time(e1),
                "finetune_loss_at_s0": float(lf0[0]), "finetune_loss_at_s_fast": float(lf1[0]),
                "s_fast_minus_s0_max": float((s_fast - dX.s).abs().max())})
    return res

# --------------------------------------------------------------------------- our arm

def main():
    if "--cpu-baseline-child" in sys.argv:
        cpu_baseline_child()
        return
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_oracle:
        cpu_base = run_cpu_baseline()          # before the first GPU call

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_04001_gb300 as P
    import synth

    # one rank per GPU; with fewer GPUs than ranks (a functional check of the N-rank
    # path with the gloo backend) ranks share devices
    local = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if args.dist_backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")

    # N ranks: one instance with N x 69,632 points, each rank its block of every point
    # class, normalised by the whole instance's counts; one all-reduce of (loss, dL/ds)
    # per step, then the replicated Adam update (weak scaling: per-rank work fixed)
    from paper_2410_04001_gb300 import shard
    net, bt = synth.workload_cdr_single(scale=world)
    model = P.lrnr_build(net.L, net.M, net.r, net.U, net.V, net.b)
    dev = torch.device("cuda", local)
    if world > 1:
        part, counts = shard.point_shard(bt, world, rank)
        db = P.DeviceBatch.from_host(part, dev, norm=counts)
    else:
        db = P.DeviceBatch.from_host(bt, dev)
    # FastLRNR construction: exact-LRNR snapshots at the 4 x 3 design plus
    # perturbations (device, FP64), EIM greedy on the device
    g = synth.rng(77)
    xs, ts = synth.snapshot_design(g, 8)
    xs_d = torch.tensor(xs, device=dev)
    ts_d = torch.tensor(ts, device=dev)
    s0 = torch.tensor(bt.s[:1], device=dev)
    rows_all = []
    for l in range(net.L):
        S = P.lrnr_snapshots(model, l, xs_d, ts_d, s0)
        rows, _, used = P.fastlrnr_select_rows(model, l, S, 16)
        rows_all.append(rows.cpu().numpy())
    n_pts = db.n_points
    P.lrnr_reserve(model, n_pts, 1)

    s = db.s.clone()
    m = torch.zeros_like(s)
    v = torch.zeros_like(s)
    step_ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    loss_out = torch.zeros(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    db_s = db.with_s(s)
    bufs = shard.partial_buffers(1, model.sum_r, model.sum_m, False, device=dev)

    def step_on(batch, s_, lo_):
        if world > 1:
            shard.sharded_spinprop_step(model, "fast", "fp32", batch, s_, m, v, step_ctr, dist,
                                        bufs=bufs, lr=1e-3, loss_out=lo_)
        else:
            P.spinprop_step(model, "fast", "fp32", batch, s_, m, v, step_ctr, 1, lr=1e-3, loss_out=lo_)

    def spin():
        step_on(db_s, s, loss_out)

    # CUDA graph of one step (2 kernels).  Kernel timing: every EVERY-th timed step runs the
    # same step eagerly with the library's timing events around the FastLRNR kernel;
    # all events are read once, after the timed region, so that the host never waits
    # for the GPU inside it (the host enqueues ahead and the GPU never idles).  Such a
    # step takes ~6 us longer than a replay (the events stand between the FastLRNR
    # kernel and the reduction it would otherwise overlap), so only every 32nd carries
    # them; the line reports both kinds of step (step_kinds).
    EVERY = 32
    for _ in range(3):
        spin()
    torch.cuda.synchronize()
    graph = None
    if world == 1:
        # (at N ranks the step holds an NCCL all-reduce and runs eagerly)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="relaxed"):
            spin()
    step_counter = [0]

    def replay():
        step_counter[0] += 1
        if graph is None or step_counter[0] % EVERY == 1:
            spin()
        else:
            graph.replay()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed_steps(fn, n, timing_model=None):
        """Run n steps, flushing L2 (256 MiB write) before each; return per-step ms
        (CUDA events on the launching stream) and the tile-kernel ms."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        if timing_model is not None:
            P.lrnr_timing_read(timing_model)      # drop earlier records
        for i in range(n):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        # the library's kernel events are read once, after the loop (no host wait inside)
        kern, kl = P.lrnr_timing_read(timing_model) if timing_model is not None else (0.0, 0)
        return [a.elapsed_time(b) for a, b in ev], kern, kl

    for _ in range(args.warmup):
        replay()
    torch.cuda.synchronize()
    P.lrnr_timing(model, True)
    P.lrnr_timing_read(model)
    step_counter[0] = 0          # the first timed step is one of the eager, event-timed ones
    try:
        gpu_id = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = ""
    clocks = ClockSampler(gpu_id)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    per_step, _, _ = timed_steps(replay, args.steps)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    kern_ms, kern_n = P.lrnr_timing_read(model)
    P.lrnr_timing(model, False)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_step = sum(per_step) / len(per_step)
    # the two kinds of timed step at N = 1: graph replays, and the eager steps that
    # carry the kernel-timing events (every EVERY-th, the first included)
    ev_steps = per_step[::EVERY]
    gr_steps = [t for i, t in enumerate(per_step) if i % EVERY]
    step_kinds = {"graph_replay_ms": sum(gr_steps) / len(gr_steps) if gr_steps else None,
                  "eager_with_kernel_events_ms": sum(ev_steps) / len(ev_steps),
                  "eager_steps": len(ev_steps)} if graph is not None else None
    if dist:
        tt = torch.tensor([ms_step], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_step = float(tt.item())
    n_total = bt.n_points                      # all ranks' points (= n_pts at N = 1)
    value = n_total / (ms_step * 1e-3)

    # ---- roofline of the dominant kernel (the fused FastLRNR kernel)
    ch = 4
    pf_int = fast_flops_per_point(net.r, [16] * net.L, ch)
    pf_bnd = fast_flops_per_point(net.r, [16] * net.L, 1)
    # this rank's launch: its own points (the whole batch at N = 1)
    flops_launch = (db.x_int.numel() * pf_int + (db.x_ic.numel() + 2 * db.t_bc.numel()) * pf_bnd)
    k_avg_ms = kern_ms / max(1, kern_n)
    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_max)
    achieved = flops_launch / (k_avg_ms * 1e-3) / 1e12
    try:
        mp = P.lrnr_measure_peaks()
    except P.LrnrError as e:
        mp = {"unavailable": str(e)}
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": K_FAST_DRAM_BYTES,
            "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu "
                             "capture of this kernel on this workload (a constant of that capture)"
                             if K_FAST_DRAM_BYTES else "no ncu capture of the current kernel yet"),
            "microbench": mp,
            "kernel": "k_fast<16,16> (fused FastLRNR residual + adjoint)",
            "kernel_ms": k_avg_ms, "flops_per_launch": flops_launch,
            "peak_note": f"FP32 FMA peak = 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz (max SM clock, {src} peaks file)"}

    # ---- variants: full-width FP32 LRNR residual + gradient, fast residual + gradient
    variants = {}
    P.lrnr_timing(model, True)
    for form, prec in (() if world > 1 else (("full", "fp32"), ("full", "bf16"), ("full", "tf32"), ("full", "bf16x3"),
                       ("fast", "fp32"), ("fast", "bf16"), ("fast", "tf32"), ("fast", "bf16x3"))):
        try:
            out = P.lrnr_residual_grad(model, form, prec, db)
        except P.LrnrError as e:
            variants[f"{form}_{prec}"] = {"unavailable": str(e)}
            continue
        torch.cuda.synchronize()
        P.lrnr_timing_read(model)
        nrep = 5 if form == "full" else 50
        ts_, km, kn = timed_steps(lambda: P.lrnr_residual_grad(model, form, prec, db, out=out), nrep, model)
        step_ms = sum(ts_) / len(ts_)
        kms = km / max(1, kn)
        fl = (bt.x_int.shape[0] * (full_flops_per_point(net.r, net.M, 4) if form == "full" else pf_int)
              + (bt.x_ic.shape[0] + 2 * bt.t_bc.shape[0]) *
              (full_flops_per_point(net.r, net.M, 1) if form == "full" else pf_bnd))
        variants[f"{form}_{prec}"] = {
            "points_per_s": n_pts / (step_ms * 1e-3), "ms_per_call": step_ms, "kernel_ms": kms,
            "tflops": fl / (kms * 1e-3) / 1e12, "frac_fp32_peak": fl / (kms * 1e-3) / 1e12 / peak,
            "hbm_gbs": (n_pts * 8) / (kms * 1e-3) / 1e9}
        if prec != "fp32":
            # executed tensor work in BF16-MMA equivalents: split-BF16 issues five BF16
            # products per contraction, a TF32 MMA runs at half the BF16 rate
            products = {"bf16": 1, "tf32": 2, "bf16x3": 5}[prec]
            variants[f"{form}_{prec}"]["frac_bf16_peak"] = (
                products * fl / (kms * 1e-3) / 1e12 / float(peaks.get("bf16_tflops", 1900.0)))
    P.lrnr_timing(model, False)

    # ---- errors against the FP64 oracle (full batch, same inputs)
    if rank == 0 and world == 1 and not args.no_oracle:
        from oracle import lrnr64, eim64

        def rel(a, b):
            a = np.asarray(a, np.float64).ravel()
            b = np.asarray(b, np.float64).ravel()
            return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        bt32 = synth.Batch(beta=f32(bt.beta), nu=f32(bt.nu), rho=f32(bt.rho), s=f32(bt.s),
                           int_off=bt.int_off, ic_off=bt.ic_off, bc_off=bt.bc_off,
                           x_int=f32(bt.x_int), t_int=f32(bt.t_int), x_ic=f32(bt.x_ic), t_bc=f32(bt.t_bc))
        # the oracle's own construction (its snapshots, its greedy); the device's rows
        # are compared with it, not fed to it
        fnet, rows_o = oracle_fast_net(P, model, net, bt.s[0], synth, torch, dev)
        for form, ref, precs in (("fast", fnet, ("fp32", "bf16", "tf32", "bf16x3")),
                                 ("full", net, ("fp32", "bf16", "tf32", "bf16x3"))):
            ro, rs, rb = lrnr64.residual_grad(ref, bt32, form)
            for prec in precs:
                if "unavailable" in variants.get(f"{form}_{prec}", {}):
                    continue
                lo, ds, dbb = P.lrnr_residual_grad(model, form, prec, db)
                variants[f"{form}_{prec}"]["err_vs_fp64_oracle"] = {
                    "loss": rel(lo.cpu(), ro), "dL_ds": rel(ds.cpu(), rs), "dL_db": rel(dbb.cpu(), rb)}
        variants["fast_fp32"]["eim_rows_match_oracle"] = all(
            np.array_equal(a, b) for a, b in zip(rows_o, rows_all))

    # ---- the larger workloads (one GPU): batched instances and the SPInProp loop
    if not args.no_configs and world == 1:
        variants.update(config_variants(P, synth, np, torch, dev, timed_steps, peak,
                                        with_oracle=(rank == 0 and not args.no_oracle)))

    # ---- end to end: host buffers in, loss and s back, through the public API.  The
    # batch arrays and s share one pinned host buffer laid out like one device buffer
    # (256-byte aligned segments), so the inputs go over in one copy; s and the loss are
    # adjacent on the device and come back in one copy.
    segs, off = {}, 0
    for k, t in db.tensors.items():
        if k == "s":
            continue
        segs[k] = (off, t)
        off += (t.numel() * t.element_size() + 255) // 256 * 256
    segs["s"] = (off, s)
    off += (s.numel() * 4 + 255) // 256 * 256
    segs["loss"] = (off, loss_out)
    off += (loss_out.numel() * 4 + 255) // 256 * 256
    hbuf = torch.zeros(off, dtype=torch.uint8).pin_memory()
    dbuf = torch.zeros(off, dtype=torch.uint8, device=dev)

    def view(buf, k):
        o, t = segs[k]
        return buf[o:o + t.numel() * t.element_size()].view(t.dtype).view(t.shape)
    for k in segs:
        view(hbuf, k).copy_(segs[k][1].detach().cpu())
    dv = {k: view(dbuf, k) for k in segs}
    db_e2e = P.DeviceBatch(db.n_inst, **{k: (dv["s"] if k == "s" else dv[k]) for k in db.tensors},
                           norm=db.norm)
    n_in = segs["s"][0] + s.numel() * 4                     # batch arrays and s
    out_lo, out_hi = segs["s"][0], segs["loss"][0] + loss_out.numel() * 4
    hout = torch.zeros(out_hi - out_lo, dtype=torch.uint8).pin_memory()
    h2d, d2h = n_in, out_hi - out_lo

    if world == 1:
        # the package's captured step with its host transfers in the same graph: one
        # replay = pinned host -> device copy, spinprop_step, device -> pinned host copy
        from paper_2410_04001_gb300.graph import SpinpropGraph
        ge2e = SpinpropGraph(model, db_e2e, dv["s"], m, v, step_ctr, 1, "fast", "fp32",
                             loss_out=dv["loss"], copy_in=[(dbuf[:n_in], hbuf[:n_in])],
                             copy_out=[(hout, dbuf[out_lo:out_hi])], lr=1e-3)
        e2e_step = ge2e.replay
    else:
        def e2e_step():
            P.lrnr_copy_pinned(dbuf[:n_in], hbuf[:n_in])
            step_on(db_e2e, dv["s"], dv["loss"])
            P.lrnr_copy_pinned(hout, dbuf[out_lo:out_hi])

    for _ in range(3):
        e2e_step()
    e_ts, _, _ = timed_steps(e2e_step, max(20, args.steps // 4))
    e2e_ms = sum(e_ts) / len(e_ts)
    if dist:
        tt = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    status = P.lrnr_last_device_status(model)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(world),
                       "form": ("FastLRNR SPInProp step (spinprop_step, 1 Adam step)" if world == 1 else
                                "FastLRNR SPInProp step on each rank's points (lrnr_residual_grad with "
                                "the instance's counts, all-reduce of loss and dL/ds, lrnr_adam_update)"),
                       "points_per_step": n_total,
                       "parallelism": f"points of one instance split over {world} ranks" if world > 1 else "single GPU",
                       "l2": "flushed before every timed step (256 MiB write)", "cuda_graph": world == 1},
            "roofline": roof,
            "cpu_baseline": cpu_base,
            "e2e": {"value": n_total / (e2e_ms * 1e-3), "unit": "points/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "note": ("one pinned host -> device copy of the batch arrays and s, "
                             + ("spinprop_step" if world == 1 else "the sharded step") +
                             ", one copy of s and the loss back to host (both copies by the "
                             "library's copy kernel, lrnr_copy_pinned)" +
                             (" (all three in one captured SpinpropGraph replay)" if world == 1
                              else ""))},
            # per SPInProp step at N = 1: the FastLRNR kernel (it computes its own tile
            # schedule for up to 4,096 instances) and the fixed-order reduction + Adam
            # kernel; at N ranks: the FastLRNR kernel, the reduction, the Adam update
            # and the step-counter kernel (the all-reduce is NCCL's)
            "gpu_launches": (2 if world == 1 else 4) * args.steps,
            "clocks": clk,
            "wall_s_timed_region": t_wall,
            "step_kinds": step_kinds,
            "device_status": status,
            "variants": variants,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
