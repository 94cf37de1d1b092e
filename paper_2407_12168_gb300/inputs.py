"""Seeded synthetic workloads for the EnSF analysis step.

This module holds no arithmetic of the method itself: it only draws the
truth fields, forecast ensembles, observations, masks and (optionally) the
pre-generated Gaussian noise that the analysis consumes.  Both the CUDA path
(through the benchmark and the tests) and the CPU oracle take their inputs
from here.  numpy only; nothing here touches a GPU.

Workloads (sizes from the paper's experiments, Sec. IV-A, and the scaled-up
cases this library is measured on):

  ``plain-64``      d = 2*64*64,  N = 20,  K = 100, H = identity on every
                    point, R = 1 (sigma_obs = 1); the paper's 64x64x2 SQG
                    accuracy setup with the entire state observed.
  ``sparse-arctan-128``  d = 2*128*128, N = 128, K = 100, a seeded 25 % of
                    points observed through arctan, sigma_obs = 0.1, prior
                    carries a smooth random bias.
  ``batched-uneven``     64 independent filters, d in {2*64^2, 2*96^2,
                    2*128^2}, N in {32, 64, 128, 256}, K = 50, 25 % arctan obs,
                    sigma_obs = 0.1.
  ``large-512``     d = 2*512*512, N = 1024, K = 100, identity obs on every
                    point, sigma_obs = 0.5.

The truth stands in for an SQG potential-temperature snapshot: a Gaussian
random field per layer whose power spectrum falls as |k|^-3 (zero mean, unit
variance per layer).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

# Stream tags: every component draws from its own seeded generator.
_TAG_TRUTH, _TAG_PRIOR, _TAG_OBS, _TAG_MASK, _TAG_BIAS, _TAG_NOISE, _TAG_SHAPES = range(7)


def rng(seed: int, tag: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(tag), int(sub)])


def gaussian_random_field(layers: int, n: int, slope: float, g: np.random.Generator,
                          std: float = 1.0) -> np.ndarray:
    """[layers][n][n] float64 field with isotropic power spectrum |k|^-slope
    (the k = 0 mode removed), each layer rescaled to standard deviation std."""
    kx = np.fft.fftfreq(n) * n
    ky = np.fft.rfftfreq(n) * n
    kk = np.sqrt(kx[:, None] ** 2 + ky[None, :] ** 2)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (-slope / 2.0)
    out = np.empty((layers, n, n))
    for layer in range(layers):
        white = g.standard_normal((n, n))
        spec = np.fft.rfft2(white) * amp
        f = np.fft.irfft2(spec, s=(n, n))
        f -= f.mean()
        f *= std / f.std()
        out[layer] = f
    return out


@dataclasses.dataclass
class Problem:
    """One analysis problem.  Arrays are float32 (uint8 for the mask) and
    C-contiguous; ``prior`` is the forecast ensemble X[n][d] row-major."""
    name: str
    n: int
    d: int
    K: int
    eps: float
    sigma_obs: float
    obs_op: int                  # 0 identity, 1 arctan
    truth: np.ndarray            # [d]
    prior: np.ndarray            # [n][d]
    y: np.ndarray                # [d] (0 where unobserved)
    mask: Optional[np.ndarray]   # [d] uint8, None = all observed
    seed: int                    # noise-stream seed
    offset: int = 0              # noise-stream offset (e.g. the cycle index)


def _problem(name, layers, grid, n, K, sigma_obs, obs_op, obs_frac, prior_std, bias_std, seed,
             eps=0.05, obs_std=None):
    d = layers * grid * grid
    truth = gaussian_random_field(layers, grid, 3.0, rng(seed, _TAG_TRUTH)).reshape(d)
    gp = rng(seed, _TAG_PRIOR)
    prior = (truth[None, :].astype(np.float32)
             + np.float32(prior_std) * gp.standard_normal((n, d), dtype=np.float32))
    if bias_std > 0.0:
        bias = gaussian_random_field(layers, grid, 5.0, rng(seed, _TAG_BIAS), std=bias_std)
        prior += bias.reshape(1, d).astype(np.float32)
    mask = None
    if obs_frac < 1.0:
        gm = rng(seed, _TAG_MASK)
        mask = np.zeros(d, dtype=np.uint8)
        mask[gm.permutation(d)[: int(round(obs_frac * d))]] = 1
    hx = np.arctan(truth) if obs_op == 1 else truth
    std = sigma_obs if obs_std is None else obs_std
    y = hx + std * rng(seed, _TAG_OBS).standard_normal(d)
    if mask is not None:
        y = np.where(mask.astype(bool), y, 0.0)
    return Problem(name=name, n=n, d=d, K=K, eps=eps, sigma_obs=float(sigma_obs), obs_op=obs_op,
                   truth=truth.astype(np.float32), prior=np.ascontiguousarray(prior),
                   y=y.astype(np.float32), mask=mask, seed=int(seed) * 1000003 + 17)


def plain_64(seed: int = 1, n: int = 20, K: int = 100) -> Problem:
    return _problem("plain-64", 2, 64, n, K, 1.0, 0, 1.0, 0.5, 0.0, seed)


def sparse_arctan_128(seed: int = 2, n: int = 128, K: int = 100) -> Problem:
    return _problem("sparse-arctan-128", 2, 128, n, K, 0.1, 1, 0.25, 0.5, 0.5, seed)


def large_512(seed: int = 4, n: int = 1024, K: int = 100) -> Problem:
    return _problem("large-512", 2, 512, n, K, 0.5, 0, 1.0, 0.5, 0.0, seed)


def medium_192(seed: int = 5, n: int = 1024, K: int = 10) -> Problem:
    """Profiling size of the large case: N = 1024, d = 2*192*192 (a 302 MB
    state, larger than L2), 10 Euler-Maruyama steps."""
    return _problem("medium-192", 2, 192, n, K, 0.5, 0, 1.0, 0.5, 0.0, seed)


def small_case(seed: int, n: int, grid: int, layers: int = 1, K: int = 10, obs_op: int = 0,
               obs_frac: float = 1.0, sigma_obs: float = 1.0, eps: float = 0.05) -> Problem:
    """A small problem for parity tests: any n, d = layers*grid*grid."""
    return _problem(f"small-n{n}-d{layers * grid * grid}", layers, grid, n, K, sigma_obs, obs_op,
                    obs_frac, 0.5, 0.0, seed, eps=eps)


def batched_uneven(seed: int = 3, count: int = 64, K: int = 50) -> List[Problem]:
    """64 independent filters with sizes drawn from the seed."""
    g = rng(seed, _TAG_SHAPES)
    grids = g.choice([64, 96, 128], size=count)
    ns = g.choice([32, 64, 128, 256], size=count)
    return [_problem(f"batched-{b}", 2, int(grids[b]), int(ns[b]), K, 0.1, 1, 0.25, 0.5, 0.5,
                     seed * 1000 + b)
            for b in range(count)]


def noise_buffer(seed: int, K: int, n: int, d: int) -> np.ndarray:
    """Pre-generated standard-normal noise xi[K+1][n][d] float32 (slice 0 is
    the initial particle sample, slice k+1 the noise of Euler-Maruyama step k)."""
    return rng(seed, _TAG_NOISE).standard_normal((K + 1, n, d), dtype=np.float32)


def unet_init_params(widths, seed: int, in_ch: int = 2, out_ch: int = 2) -> np.ndarray:
    """Seeded initial parameters of the U-Net surrogate (flat order of the
    library): He-uniform convolution weights, zero biases, a small head."""
    g = rng(seed, _TAG_SHAPES, 99)
    c1, c2, c3, c4 = widths
    convs = [(in_ch, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3), (c3, c4), (c4, c4),
             (c4 + c3, c3), (c3, c3), (c3 + c2, c2), (c2, c2), (c2 + c1, c1), (c1, c1)]
    parts = []
    for ci, co in convs:
        bound = np.sqrt(6.0 / (9 * ci))
        parts.append(g.uniform(-bound, bound, 9 * ci * co))
        parts.append(np.zeros(co))
    parts.append(g.uniform(-0.01, 0.01, c1 * out_ch))
    parts.append(np.zeros(out_ch))
    return np.concatenate(parts).astype(np.float32)


WORKLOADS = {
    "plain-64": plain_64,
    "sparse-arctan-128": sparse_arctan_128,
    "large-512": large_512,
    "medium-192": medium_192,
}
