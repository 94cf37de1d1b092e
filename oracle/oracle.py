"""FP64 CPU oracle of the EnSF analysis step -- Python loader.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library and
its Python binding never import, link or execute anything under ``oracle/``.

The arithmetic lives in ``ensf_oracle.c`` (plain C99, FP64, OpenMP over
members); this module compiles it with gcc on demand and marshals numpy arrays.
Every function cites the passage of the paper it follows (Sec. III-A).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ensf_oracle.c")
_LIB = os.path.join(_HERE, "libensf_oracle.so")
_lock = threading.Lock()
_lib = None

OBS_IDENTITY = 0
OBS_ARCTAN = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE semantics kept: no fast-math and
    no FMA contraction, so x86 and Arm hosts evaluate the same expressions)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.ensf_oracle_schedule.argtypes = [ctypes.c_double, ctypes.c_double, dp]
        lib.ensf_oracle_schedule.restype = None
        lib.ensf_oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.ensf_oracle_philox4x32_10.restype = None
        lib.ensf_oracle_noise.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int64]
        lib.ensf_oracle_noise.restype = ctypes.c_double
        lib.ensf_oracle_noise_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int64, dp]
        lib.ensf_oracle_noise_fill.restype = None
        lib.ensf_oracle_lik_score.argtypes = [dp, fp, u8p, ctypes.c_int64, ctypes.c_double,
                                              ctypes.c_int, dp]
        lib.ensf_oracle_lik_score.restype = None
        lib.ensf_oracle_weights.argtypes = [fp, ctypes.c_int, ctypes.c_int64, dp, ctypes.c_double,
                                            ctypes.c_double, dp, dp]
        lib.ensf_oracle_weights.restype = None
        lib.ensf_oracle_prior_score.argtypes = [fp, ctypes.c_int, ctypes.c_int64, dp,
                                                ctypes.c_double, ctypes.c_double, dp]
        lib.ensf_oracle_prior_score.restype = None
        lib.ensf_oracle_analysis.argtypes = [fp, ctypes.c_int, ctypes.c_int64, fp, u8p,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, fp, ctypes.c_uint64, ctypes.c_uint32,
                                             ip, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_uint64, dp, dp, dp]
        lib.ensf_oracle_analysis.restype = ctypes.c_int
        lib.ensf_oracle_mean_rmse.argtypes = [dp, ctypes.c_int, ctypes.c_int64, fp, dp]
        lib.ensf_oracle_mean_rmse.restype = ctypes.c_double
        lib.ensf_oracle_num_threads.argtypes = []
        lib.ensf_oracle_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().ensf_oracle_num_threads())


def schedule(t: float, eps: float) -> dict:
    """Eq. 9 drift/diffusion with alpha_t = 1 - t(1-eps), beta_t^2 = t, and the
    damping h(t) = 1 - t of Eq. 11."""
    out = np.zeros(5)
    _load().ensf_oracle_schedule(float(t), float(eps), _ptr(out, ctypes.c_double))
    return dict(alpha=out[0], beta2=out[1], b=out[2], sigma2=out[3], h=out[4])


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _load().ensf_oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                                      _ptr(o, ctypes.c_uint32))
    return o


def noise(seed: int, offset: int, k: int, i: int, d: int) -> np.ndarray:
    """Row xi[k][i][0:d] of the counter-based standard-normal stream."""
    out = np.zeros(d)
    _load().ensf_oracle_noise_fill(seed, offset, k, i, d, _ptr(out, ctypes.c_double))
    return out


def lik_score(z, y, mask, sigma_obs: float, obs_op: int) -> np.ndarray:
    """grad_z log P(y|z) of Eq. 5 (with the one half), R = sigma_obs^2 I."""
    z = _f64(z)
    y = _f32(y)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    g = np.zeros_like(z)
    _load().ensf_oracle_lik_score(_ptr(z, ctypes.c_double), _ptr(y, ctypes.c_float),
                                  _ptr(m, ctypes.c_uint8), z.size, float(sigma_obs), int(obs_op),
                                  _ptr(g, ctypes.c_double))
    return g


def weights(X, z, alpha: float, beta2: float):
    """Normalised Monte-Carlo weights of Eq. 16 and the log-kernels of Eq. 12."""
    X = _f32(X)
    z = _f64(z)
    n, d = X.shape
    w = np.zeros(n)
    logit = np.zeros(n)
    _load().ensf_oracle_weights(_ptr(X, ctypes.c_float), n, d, _ptr(z, ctypes.c_double),
                                float(alpha), float(beta2), _ptr(w, ctypes.c_double),
                                _ptr(logit, ctypes.c_double))
    return w, logit


def prior_score(X, z, alpha: float, beta2: float) -> np.ndarray:
    """Monte-Carlo prior score of Eq. 15."""
    X = _f32(X)
    z = _f64(z)
    n, d = X.shape
    s = np.zeros(d)
    _load().ensf_oracle_prior_score(_ptr(X, ctypes.c_float), n, d, _ptr(z, ctypes.c_double),
                                    float(alpha), float(beta2), _ptr(s, ctypes.c_double))
    return s


def analysis(X, y, mask, sigma_obs: float, K: int, eps: float, obs_op: int = OBS_IDENTITY,
             noise_buf=None, seed: int = 0, offset: int = 0, rows=None, k_stop=None,
             return_traj: bool = False, return_diag: bool = False, logit_perturb: float = 0.0,
             perturb_seed: int = 0, perm=None, J=None):
    """Run the EnSF analysis (Eq. 7 discretised by Euler-Maruyama with the
    score of Eq. 17) for the particle rows ``rows`` (default: all).

    Returns ``out`` [len(rows)][d] float64; with ``return_traj`` also the
    trajectory [k_stop+1][len(rows)][d]; with ``return_diag`` also
    [k_stop][len(rows)][2] = (top-two log-kernel gap, log-kernel error scale)
    per step and row.  ``logit_perturb`` > 0 (tests of conditioning only)
    adds +/- logit_perturb * alpha |z_i| |x_j| / beta^2 to every log-kernel.
    ``perm``, ``J``: mini-batch prior score over the window k mod (n/J) of J
    members of the permutation (Eq. 15-16 with J < N)."""
    X = _f32(X)
    n, d = X.shape
    y = _f32(y)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    nb = _f32(noise_buf)
    if nb is not None and nb.shape != (K + 1, n, d):
        raise ValueError(f"noise buffer must be [K+1][n][d] = {(K + 1, n, d)}, got {nb.shape}")
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    nrows = n if r is None else r.size
    ks = K if k_stop is None else int(k_stop)
    out = np.zeros((nrows, d))
    traj = np.zeros((ks + 1, nrows, d)) if return_traj else None
    diag = np.zeros((ks, nrows, 2)) if return_diag else None
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    jj = n if J is None else int(J)
    rc = _load().ensf_oracle_analysis(
        _ptr(X, ctypes.c_float), n, d, _ptr(y, ctypes.c_float), _ptr(m, ctypes.c_uint8),
        float(sigma_obs), int(K), float(eps), int(obs_op), _ptr(nb, ctypes.c_float),
        int(seed), int(offset), _ptr(r, ctypes.c_int), nrows, ks, _ptr(pm, ctypes.c_int), jj,
        float(logit_perturb), int(perturb_seed),
        _ptr(out, ctypes.c_double), _ptr(traj, ctypes.c_double), _ptr(diag, ctypes.c_double))
    if rc != 0:
        raise ValueError("ensf_oracle_analysis rejected its arguments")
    res = [out] + ([traj] if return_traj else []) + ([diag] if return_diag else [])
    return res[0] if len(res) == 1 else tuple(res)


def mean_rmse(Z, truth):
    """FP64 ensemble mean over rows and the RMSE of that mean against truth."""
    Z = _f64(Z)
    truth = _f32(truth)
    n, d = Z.shape
    mean = np.zeros(d)
    rmse = _load().ensf_oracle_mean_rmse(_ptr(Z, ctypes.c_double), n, d,
                                         _ptr(truth, ctypes.c_float), _ptr(mean, ctypes.c_double))
    return mean, float(rmse)


def model_error(state, coef, seed: int, cycle: int) -> np.ndarray:
    """Imperfect-model error of the twin experiment (Sec. IV-A): additive
    Gaussian errors, uncorrelated in space (diagonal covariance) and white in
    time, made of several stochastic processes, each realised or not in a
    given forecast interval.  The caller folds each process's realisation
    (drawn as an input), amplitude and the model's mean value into coef[p];
    the result is

        state[b][j] + sum_p coef[p] * xi_p[b][j],

    xi_p[b][j] = noise(seed, offset = cycle, k = p, particle b, element j),
    the standard normal of the same counter-based stream as the analysis
    noise, in FP64."""
    x = np.array(state, dtype=np.float64, copy=True)
    if x.ndim == 1:
        x = x[None, :]
    B, d = x.shape
    for p, c in enumerate(coef):
        if c != 0.0:
            for b in range(B):
                x[b] += float(c) * noise(seed, cycle, p, b, d)
    return x


def relax_spread(prior, z, factor: float, mode: str = "spread") -> np.ndarray:
    """Relaxation of the analysis ensemble toward the forecast ensemble after
    each cycled analysis (Sec. IV-A: the analysis spread is relaxed to the
    prior values), per state variable over the n members, in FP64.

    "spread" (relaxation to prior spread, Whitaker and Hamill 2012): the
    analysis anomalies z_i - mean(z) are scaled by (1 - a) + a s_f / s_a, s_f and
    s_a the forecast and analysis standard deviations (factor 1 where s_a = 0).
    "perturbations" (relaxation to prior perturbations, Zhang et al. 2004):
    the anomalies become (1 - a)(z_i - mean(z)) + a (x_i - mean(x)).
    The analysis mean is kept in both."""
    x = np.asarray(prior, dtype=np.float64)
    za = np.asarray(z, dtype=np.float64)
    ma, mf = za.mean(axis=0), x.mean(axis=0)
    da, df = za - ma, x - mf
    if mode == "perturbations":
        return ma + (1.0 - factor) * da + factor * df
    sa, sf = np.sqrt((da ** 2).mean(axis=0)), np.sqrt((df ** 2).mean(axis=0))
    ratio = np.divide(sf, sa, out=np.ones_like(sa), where=sa > 0)
    return ma + da * ((1.0 - factor) + factor * ratio)

