"""Writes ``large512_subsample64.npz``: the FP64 oracle's analysis of 64 member
rows of the large-512 workload (N = 1024, d = 2 x 512 x 512, K = 100,
identity observations of every point with sigma_obs = 0.5), for the
ensemble-RMSE check on a member subsample of the big configuration.

The oracle's analysis is exact on any subset of rows (each particle evolves
given X, y and its own noise draws only), so the 64 rows need not be
recomputed with the rest of the ensemble.  Stored, per row: the values at
4096 seeded state indices and the row norm; the FP64 ensemble mean of the 64
rows as its RMSE against the truth; and, per row, the smallest ratio over
the K steps of the oracle's top-two log-kernel gap to its log-kernel error
scale (rows with a small ratio sit near a tie between forecast members).

Uses only ``oracle/`` and the seeded input generators.  On 8 host cores it
runs for about an hour:  python tests/golden/make_large512_subsample.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as o  # noqa: E402
from paper_2407_12168_gb300 import inputs  # noqa: E402

ROWS = np.arange(0, 1024, 16, dtype=np.int32)  # 64 members spread over the ensemble
N_IDX = 4096
IDX_SEED = 20240716


def main() -> None:
    p = inputs.large_512()
    t0 = time.time()
    out, diag = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed,
                           offset=p.offset, rows=ROWS, return_diag=True)
    secs = time.time() - t0
    idx = np.sort(np.random.default_rng(IDX_SEED).choice(p.d, size=N_IDX, replace=False)).astype(np.int64)
    truth = p.truth.astype(np.float32).astype(np.float64)
    mean = out.mean(axis=0)
    rmse = float(np.sqrt(np.mean((mean - truth) ** 2)))
    gap_ratio = (diag[:, :, 0] / np.maximum(diag[:, :, 1], 1e-300)).min(axis=0)
    np.savez_compressed(os.path.join(HERE, "large512_subsample64.npz"), rows=ROWS, idx=idx,
                        values=out[:, idx], row_norm=np.linalg.norm(out, axis=1), rmse=rmse,
                        gap_ratio=gap_ratio, seconds=secs, threads=o.num_threads())
    print(f"64 rows in {secs:.0f} s on {o.num_threads()} threads; subsample RMSE {rmse:.7f}")


if __name__ == "__main__":
    main()
