"""Well-formedness of the stored oracle outputs under tests/golden/ (CPU).

The values themselves come from the oracle (the committed script beside
them); these checks only guard the files against truncation or a mismatched
workload before a GPU test relies on them."""
import os

import numpy as np
import pytest

from paper_2407_12168_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_large512_subsample_is_well_formed():
    path = os.path.join(GOLDEN, "large512_subsample64.npz")
    if not os.path.exists(path):
        pytest.skip("written by tests/golden/make_large512_subsample.py")
    g = np.load(path)
    d = 2 * 512 * 512
    rows, idx, vals = g["rows"], g["idx"], g["values"]
    assert rows.shape == (64,) and (np.diff(rows) > 0).all() and rows[-1] < 1024
    assert idx.shape == (4096,) and (np.diff(idx) > 0).all() and 0 <= idx[0] and idx[-1] < d
    assert vals.shape == (64, 4096) and np.isfinite(vals).all()
    assert g["row_norm"].shape == (64,)
    # a subset of a row's entries cannot carry more than the whole row
    assert (np.linalg.norm(vals, axis=1) <= g["row_norm"] * (1 + 1e-12)).all()
    # sampled entries carry about 4096/d of each row's energy
    frac = (np.linalg.norm(vals, axis=1) / g["row_norm"]) ** 2
    assert np.all(np.abs(frac / (4096 / d) - 1) < 0.3)
    assert np.isfinite(float(g["rmse"])) and float(g["rmse"]) > 0
    assert g["gap_ratio"].shape == (64,) and (g["gap_ratio"] >= 0).all()


def test_large512_workload_matches_the_stored_subsample_recipe():
    """The workload the stored rows were computed for: N = 1024, d = 2 x
    512^2, K = 100, identity observations, sigma_obs = 0.5, eps = 0.05."""
    p = inputs.large_512.__defaults__
    assert p == (4, 1024, 100)
