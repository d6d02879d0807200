"""Write ``oracle_small.json``: the FP64 oracle's per-instance loss, dL/ds and dL/db on a
small seeded case, for the full-width LRNR (Eq. 2.1-2.2) and the FastLRNR (Eq. 2.8,
rows and bases from the greedy EIM of Sec. 2.2), under the MSE (Eq. 3.5) and l1
(Eq. 3.6) losses of the CDR problem (Eq. 4.1).

The file is a regression snapshot of the oracle: every value in it comes from
``oracle/`` on inputs drawn by ``synth``; nothing comes from the CUDA path.  The test
``tests/test_oracle_golden.py`` recomputes it and compares, so a change to the
oracle's arithmetic shows up as a failing test.

    python tests/golden/make_golden.py      (from the repository root)
"""
from __future__ import annotations

import json
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

import synth  # noqa: E402
from oracle import eim64, lrnr64  # noqa: E402

OUT = Path(__file__).with_name("oracle_small.json")
CASE = {"seed": 2410, "L": 3, "M": 12, "r": 3, "rhat": 5, "n_int": [24, 0, 17], "n_ic": [6, 4, 0],
        "n_bc": [3, 0, 5], "beta": [5.0, 0.0, 2.0], "nu": [1.0, 0.0, 0.5], "rho": [2.0, 1.0, 0.0]}


def compute() -> dict:
    c = CASE
    g = synth.rng(c["seed"])
    net = synth.make_net(g, L=c["L"], M=c["M"], r=c["r"])
    bt = synth.make_batch(g, net, c["n_int"], c["n_ic"], c["n_bc"], c["beta"], c["nu"], c["rho"])
    xs, ts = synth.snapshot_design(g, 4)
    rows, Xis = [], []
    for l in range(net.L):
        p, Xi, _ = eim64.eim_greedy(lrnr64.hidden_states(net, bt.s[0], xs, ts, l), c["rhat"], 0.0)
        rows.append(p)
        Xis.append(Xi)
    fnet = lrnr64.make_fast(net, rows, Xis)
    out = {"case": c, "rows": [np.asarray(p).tolist() for p in rows]}
    for form, model in (("full", net), ("fast", fnet)):
        for loss in ("mse", "l1"):
            lo, ds, db = lrnr64.residual_grad(model, bt, form, loss=loss)
            out[f"{form}_{loss}"] = {"loss": np.asarray(lo).tolist(), "dL_ds": np.asarray(ds).tolist(),
                                     "dL_db": np.asarray(db).tolist()}
    return out


def main():
    d = compute()
    OUT.write_text("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in d.items())
                   + "\n}\n")
    print(f"wrote {OUT.relative_to(ROOT)}")


if __name__ == "__main__":
    main()
