"""The oracle against its stored FP64 snapshot (``tests/golden/oracle_small.json``,
written by ``tests/golden/make_golden.py`` from the oracle alone): a change to the
oracle's arithmetic fails here until the snapshot is rewritten."""
import importlib.util
import json
from pathlib import Path

import numpy as np

GOLDEN = Path(__file__).with_name("golden")


def _load_maker():
    spec = importlib.util.spec_from_file_location("make_golden", GOLDEN / "make_golden.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_matches_its_stored_snapshot():
    stored = json.loads((GOLDEN / "oracle_small.json").read_text())
    now = _load_maker().compute()
    assert now["case"] == stored["case"]
    assert now["rows"] == stored["rows"]                   # EIM rows: exact
    for key in ("full_mse", "full_l1", "fast_mse", "fast_l1"):
        for q in ("loss", "dL_ds", "dL_db"):
            a, b = np.asarray(now[key][q]), np.asarray(stored[key][q])
            assert a.shape == b.shape, (key, q)
            # summation order may differ between BLAS builds: rounding-level tolerance
            assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b))), (key, q)
