"""Shared helpers of the GPU parity tests: run the oracle and the CUDA path on
the same seeded inputs and compare member by member.

Tolerance (per member i, relative L2 over the state vector):
  * FP32 and split-BF16x3 paths: |z_gpu - z_ref| / |z_ref| <= 1e-4
  * paths with a plain BF16 contraction: <= 1e-2
  * ensemble-mean RMSE against truth within 1 % of the oracle's.

Near-tie clause: the weights of Eq. 16 are a softmax of log-kernels, and the
GPU forms them in the expanded form (2 alpha z.x - alpha^2 |x|^2)/(2 beta^2),
whose rounding error is a fraction eps_path of alpha |z| |x| / beta^2 (eps_path
= the relative accuracy of one dot product z . x_j on that path).  A particle
whose leading weights are nearly tied at some step turns that error into a
visible change of its result.  Whether a member's result is determined to the
tolerance at the GPU path's accuracy is measured on the oracle itself: it is
re-run with every log-kernel perturbed by +/- eps_path alpha |z| |x| / beta^2
(two sign patterns); a member whose oracle result moves by more than half the
tolerance is ill-conditioned ("near tie").  Such members are counted and
reported, never silently dropped; each test bounds their number.

eps_path (typical error of a length-d dot product, as a fraction of |z||x|):
  FP32 CUDA cores    2 * 2^-24
  split-BF16x3       3 * 2^-18 / sqrt(d) + 2 * 2^-24   (operands carried to
                     ~16 bits: residuals of the two-term split and the dropped
                     lo*lo product, random in sign across the d terms)
  BF16               2 * 2^-9 / sqrt(d)
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as o

TOL_FP32 = 1e-4
TOL_BF16 = 1e-2


def eps_path(prec: str, d: int) -> float:
    if prec == "fp32":
        return 2.0 * 2.0 ** -24
    if prec == "split":
        return 3.0 * 2.0 ** -18 / np.sqrt(d) + 2.0 * 2.0 ** -24
    if prec == "tf32":  # operands rounded to TF32 (10 stored mantissa bits)
        return 2.0 * 2.0 ** -11 / np.sqrt(d) + 2.0 * 2.0 ** -24
    return 2.0 * 2.0 ** -9 / np.sqrt(d)


def run_oracle(p, rows=None, noise_buf=None, logit_perturb=0.0, perturb_seed=0, perm=None, J=None):
    return o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, noise_buf=noise_buf,
                      seed=p.seed, offset=p.offset, rows=rows, logit_perturb=logit_perturb,
                      perturb_seed=perturb_seed, perm=perm, J=J)


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def conditioning(p, ref, rows=None, noise_buf=None, prec="fp32", perm=None, J=None):
    """Largest relative change of each oracle member under log-kernel
    perturbations of the size the GPU path's Gram leaves (two sign patterns)."""
    eps = eps_path(prec, p.d)
    return np.maximum.reduce([_rel(run_oracle(p, rows=rows, noise_buf=noise_buf, logit_perturb=eps,
                                              perturb_seed=s, perm=perm, J=J), ref) for s in (1, 2)])


def compare_members(gpu: np.ndarray, ref: np.ndarray, cond: np.ndarray, tol: float):
    """Returns (rel_err [m], near_tie [m], failing [m])."""
    rel = _rel(gpu.astype(np.float64), ref)
    near_tie = cond > 0.5 * tol
    failing = (rel > tol) & ~near_tie
    return rel, near_tie, failing


def describe(rel, near_tie, failing) -> str:
    return (f"max rel err {rel.max():.3e} (median {np.median(rel):.3e}); near-tie members "
            f"{int(near_tie.sum())}; failing {np.flatnonzero(failing).tolist()[:10]}")
