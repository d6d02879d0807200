"""Checkpoint and resume of a SPInProp run: the coefficients s, the Adam moments and
step counter, and the reduced network (EIM rows P and bases Xi per hidden layer),
saved as one .npz.  Loading reinstalls the reduced layers in a model built from the
same bases (``fastlrnr_select_rows`` with given rows and Xi), after which
``spinprop_step`` continues exactly as the uninterrupted run would (same GPU, same
launch shapes).  The paper hands the trained s_fast to the full network (Sec. 3.2);
this is the host-side state that makes that hand-off and a restart possible."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def save(path, s, m, v, step, rows, Xis):
    """rows[l] (rhat_l,) int and Xis[l] (rhat_l, M) float64 per hidden layer, as
    ``fastlrnr_select_rows`` returns them (device or host); s, m, v (n_inst, sum_r)
    and the step counter (1-element int64)."""
    host = lambda t: t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)
    arrays = {"s": host(s), "m": host(m), "v": host(v), "step": host(step).astype(np.int64),
              "n_layers": np.array(len(rows), np.int64)}
    for l, (r, X) in enumerate(zip(rows, Xis)):
        arrays[f"rows{l}"] = host(r).astype(np.int32)
        arrays[f"xi{l}"] = host(X).astype(np.float64)
    np.savez(path, **arrays)


def load(path, model: B.Model, device="cuda"):
    """Reinstall the reduced layers in ``model`` and return device tensors
    (s, m, v, step) ready for ``spinprop_step``."""
    z = np.load(path)
    for l in range(int(z["n_layers"])):
        rows = torch.tensor(z[f"rows{l}"], device=device)
        xi = torch.tensor(np.ascontiguousarray(z[f"xi{l}"]), device=device)
        B.fastlrnr_select_rows(model, l, rhat=rows.numel(), rows_in=rows, Xi_in=xi)
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device=device)
    return (dev(z["s"], torch.float32), dev(z["m"], torch.float32), dev(z["v"], torch.float32),
            dev(z["step"], torch.int64))
