"""Launch-shape autotuner for the SIMT tile kernels.

For a given model, batch, form and precision it times each candidate shape
(points per tile, cap on resident CTAs per SM) with the library's own CUDA-event
timing of the tile kernel, keeps the fastest, installs it with
``lrnr_set_tuning`` and caches the choice in a JSON file keyed by the problem
shape, so later processes reuse it without timing again.
"""
from __future__ import annotations

import json
import os

import torch

from . import binding as B

CANDIDATES = {
    "fast": [(nt, cta) for nt in (128, 64) for cta in (0, 2, 1)],
    "full": [(nt, cta) for nt in (64, 32) for cta in (0, 2, 1)],
}


def _key(model, batch, form, prec):
    info = B.lrnr_model_info(model)
    pts = batch.n_points
    bucket = 1 << max(0, (pts - 1).bit_length())          # power-of-two point bucket
    return f"{form}/{prec}/L{info['L']}/M{info['M']}/sr{info['sum_r']}/n{batch.n_inst}/p{bucket}"


def _time(model, batch, form, prec, reps):
    out = B.lrnr_residual_grad(model, form, prec, batch)
    torch.cuda.synchronize()
    B.lrnr_timing(model, True)
    for _ in range(reps):
        B.lrnr_residual_grad(model, form, prec, batch, out=out)
    ms, n = B.lrnr_timing_read(model)
    B.lrnr_timing(model, False)
    return ms / max(1, n)


def autotune(model, batch, form="fast", prec="fp32", cache=None, reps=5):
    """Pick and install the fastest shape; returns {"nt", "ctas_per_sm", "ms", "key"}."""
    if form == "full" and prec != "fp32":
        return {"nt": 128, "ctas_per_sm": 1, "ms": None, "key": None}   # fixed tensor-core shape
    cache = cache or os.path.join(os.path.expanduser("~"), ".cache", "lrnr_autotune.json")
    key = _key(model, batch, form, prec)
    table = {}
    if os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table:
        best = table[key]
        B.lrnr_set_tuning(model, form, prec, best["nt"], best["ctas_per_sm"])
        return dict(best, key=key)
    results = []
    for nt, cta in CANDIDATES[form]:
        B.lrnr_set_tuning(model, form, prec, nt, cta)
        results.append((_time(model, batch, form, prec, reps), nt, cta))
    ms, nt, cta = min(results)
    B.lrnr_set_tuning(model, form, prec, nt, cta)
    best = {"nt": nt, "ctas_per_sm": cta, "ms": ms,
            "timings": [{"nt": n, "ctas_per_sm": c, "ms": t} for t, n, c in results]}
    table[key] = best
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    except OSError:
        pass
    return dict(best, key=key)
