"""Python binding of the EnSF C ABI (``include/ensf.h``).

Argument marshalling only: every step of the analysis runs in the CUDA
library ``_lib/libensf.so``.  PyTorch provides device memory and the current
stream.  There is no CPU fallback: if the library cannot be built or loaded,
or no CUDA device is present, every call raises.
"""
from __future__ import annotations

import ctypes
import threading
from typing import Optional

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, EUNSUPPORTED = range(7)
OBS_IDENTITY, OBS_ARCTAN = 0, 1
PREC_FP32, PREC_SPLIT_BF16X3, PREC_BF16 = 0, 1, 2
FLAG_CHECK_FINITE = 1
FLAG_CUDA_GRAPH = 2
FLAG_PERSISTENT = 8
FLAG_INLINE_NOISE = 4
FLAG_WX_UNSTAGED = 16

PREC_TF32 = 3
PRECISIONS = {"fp32": PREC_FP32, "split": PREC_SPLIT_BF16X3, "bf16": PREC_BF16, "tf32": PREC_TF32}


class EnsfConfig(ctypes.Structure):
    _fields_ = [("max_n", ctypes.c_int), ("max_d", ctypes.c_int64), ("gram", ctypes.c_int),
                ("wx", ctypes.c_int), ("flags", ctypes.c_uint)]


class EnsfNoise(ctypes.Structure):
    _fields_ = [("buf", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("offset", ctypes.c_uint32)]


class EnsfInstance(ctypes.Structure):
    _fields_ = [("prior", ctypes.c_void_p), ("n", ctypes.c_int), ("d", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("obs_mask", ctypes.c_void_p), ("obs_op", ctypes.c_int), ("sigma_obs", ctypes.c_float),
                ("noise", EnsfNoise), ("out", ctypes.c_void_p)]


class EnsfShard(ctypes.Structure):
    _fields_ = [("prior", ctypes.c_void_p), ("n", ctypes.c_int), ("d_local", ctypes.c_int64),
                ("col0", ctypes.c_int64), ("y", ctypes.c_void_p), ("obs_mask", ctypes.c_void_p),
                ("obs_op", ctypes.c_int), ("sigma_obs", ctypes.c_float), ("K", ctypes.c_int),
                ("eps", ctypes.c_float), ("noise", EnsfNoise), ("out", ctypes.c_void_p)]


class EnsfProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("timed_launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class EnsfTuning(ctypes.Structure):
    _fields_ = [("gram_tile_n", ctypes.c_int), ("gram_stages", ctypes.c_int), ("gram_splits", ctypes.c_int),
                ("gram_ms", ctypes.c_float), ("wx_tile_n", ctypes.c_int), ("wx_ms", ctypes.c_float),
                ("gram_k_block", ctypes.c_int), ("gram_cta_pair", ctypes.c_int),
                ("gram_noise_warps", ctypes.c_int), ("gram_fp32_particles", ctypes.c_int),
                ("noise_inline", ctypes.c_int), ("pdl", ctypes.c_int), ("gram_fused_softmax", ctypes.c_int)]


class EnsfSqgParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("L", ctypes.c_double), ("H", ctypes.c_double), ("N_over_f", ctypes.c_double),
                ("shear", ctypes.c_double), ("dt", ctypes.c_double), ("tau_diss", ctypes.c_double),
                ("diffusion", ctypes.c_int), ("tau_relax", ctypes.c_double)]


class EnsfUnetConfig(ctypes.Structure):
    _fields_ = [("in_ch", ctypes.c_int), ("out_ch", ctypes.c_int), ("widths", ctypes.c_int * 4),
                ("height", ctypes.c_int), ("width", ctypes.c_int), ("max_batch", ctypes.c_int)]


class EnsfError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


# (name, restype, argtypes) of every exported entry point
_SIGNATURES = [
    ("ensf_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(EnsfConfig)]),
    ("ensf_create", ctypes.c_int, [ctypes.POINTER(EnsfConfig), ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    ("ensf_analysis", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_int, ctypes.c_float, ctypes.POINTER(EnsfNoise),
                                     ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_analysis_minibatch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                               ctypes.c_int, ctypes.c_float, ctypes.POINTER(EnsfNoise),
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_float, ctypes.POINTER(EnsfNoise), ctypes.c_void_p,
                                     ctypes.POINTER(EnsfTuning), ctypes.c_void_p]),
    ("ensf_batch_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(EnsfConfig), ctypes.POINTER(EnsfInstance),
                                                     ctypes.c_int]),
    ("ensf_analysis_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EnsfInstance), ctypes.c_int,
                                             ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.c_void_p]),
    ("ensf_autotune_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EnsfInstance), ctypes.c_int,
                                             ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                             ctypes.c_void_p]),
    ("ensf_set_batch_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ensf_shard_splits", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int)]),
    ("ensf_shard_prep", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EnsfShard), ctypes.c_void_p,
                                       ctypes.c_void_p]),
    ("ensf_shard_gram", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EnsfShard), ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    ("ensf_shard_update", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EnsfShard), ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_weights", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_weights_static", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    ("ensf_philox_normal", ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_row_norms", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    ("ensf_relax_spread", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                         ctypes.c_float, ctypes.c_int, ctypes.c_void_p]),
    ("ensf_selftest_timeouts", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_set_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(EnsfTuning)]),
    ("ensf_model_error", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_float),
                                        ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]),
    ("ensf_stats_scratch_bytes", ctypes.c_size_t, [ctypes.c_int64]),
    ("ensf_ensemble_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    ("ensf_profile_enable", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ensf_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EnsfProfileEntry), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    ("ensf_sqg_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(EnsfSqgParams), ctypes.c_int]),
    ("ensf_sqg_create", ctypes.c_int, [ctypes.POINTER(EnsfSqgParams), ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    ("ensf_sqg_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("ensf_sqg_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("ensf_unet_param_count", ctypes.c_int64, [ctypes.POINTER(EnsfUnetConfig)]),
    ("ensf_unet_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(EnsfUnetConfig)]),
    ("ensf_unet_create", ctypes.c_int, [ctypes.POINTER(EnsfUnetConfig), ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("ensf_unet_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_unet_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_unet_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    ("ensf_unet_gradients", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_unet_train_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_unet_get_moments", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    ("ensf_unet_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("ensf_host_alloc", ctypes.c_int, [ctypes.c_size_t, ctypes.c_uint, ctypes.POINTER(ctypes.c_void_p)]),
    ("ensf_host_free", ctypes.c_int, [ctypes.c_void_p]),
    ("ensf_copy_sm", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                    ctypes.c_void_p]),
    ("ensf_host_registered", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("ensf_host_huge_fraction", ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)]),
    ("ensf_host_numa", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("ensf_status_sync", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ensf_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("ensf_last_error", ctypes.c_char_p, []),
    ("ensf_destroy", ctypes.c_int, [ctypes.c_void_p]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load (building first if needed) the CUDA library and declare signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        lib = ctypes.CDLL(path)
        for name, res, args in _SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, where: str) -> None:
    if status != OK:
        lib = load()
        raise EnsfError(status, where, lib.ensf_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the EnSF library needs a CUDA device; none is available")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Filter:
    """An EnSF handle plus its device workspace (a torch uint8 tensor).

    ``gram`` and ``wx`` choose the arithmetic of the Gram Z X^T and of the
    weighted sum W X: ``"fp32"`` (CUDA cores), ``"split"`` (BF16x3 on tensor
    cores), ``"bf16"`` (one BF16 product on tensor cores) or, for the Gram
    only, ``"tf32"`` (tensor cores on the FP32 centred operands).  ``persistent``:
    with FP32 precisions and n <= 128, all K steps run in one cooperative
    launch (small filters)."""

    def __init__(self, max_n: int, max_d: int, gram: str = "fp32", wx: str = "fp32",
                 check_finite: bool = False, graph: bool = False, inline_noise: bool = False,
                 persistent: bool = False, wx_unstaged: bool = False):
        torch = _torch()
        lib = load()
        self.cfg = EnsfConfig(int(max_n), int(max_d), PRECISIONS[gram], PRECISIONS[wx],
                              (FLAG_CHECK_FINITE if check_finite else 0) | (FLAG_CUDA_GRAPH if graph else 0)
                              | (FLAG_INLINE_NOISE if inline_noise else 0) | (FLAG_PERSISTENT if persistent else 0)
                              | (FLAG_WX_UNSTAGED if wx_unstaged else 0))
        nbytes = lib.ensf_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise ValueError("invalid EnSF configuration")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(lib.ensf_create(ctypes.byref(self.cfg), ctypes.c_void_p(aligned), nbytes, ctypes.byref(h)),
               "ensf_create")
        self._h = h
        self.gram, self.wx = gram, wx

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ensf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def analysis(self, prior, y, mask, sigma_obs: float, K: int, eps: float, obs_op: int = OBS_IDENTITY,
                 seed: int = 0, offset: int = 0, noise=None, out=None, stream=None):
        """Run the analysis step; returns ``out`` [n][d] (allocated if None)."""
        torch = _torch()
        _dev(prior, torch.float32, "prior")
        n, d = prior.shape
        _dev(y, torch.float32, "y")
        if mask is not None:
            _dev(mask, torch.uint8, "mask")
        if noise is not None:
            _dev(noise, torch.float32, "noise")
            if tuple(noise.shape) != (K + 1, n, d):
                raise ValueError(f"noise must have shape {(K + 1, n, d)}")
        if out is None:
            out = torch.empty_like(prior)
        _dev(out, torch.float32, "out")
        nz = EnsfNoise(noise.data_ptr() if noise is not None else None, int(seed) & (2 ** 64 - 1),
                       int(offset) & 0xFFFFFFFF)
        st = load().ensf_analysis(self._h, prior.data_ptr(), n, d, y.data_ptr(),
                                  mask.data_ptr() if mask is not None else None, int(obs_op),
                                  float(sigma_obs), int(K), float(eps), ctypes.byref(nz), out.data_ptr(),
                                  _stream_ptr(stream))
        _check(st, "ensf_analysis")
        return out

    def analyses_from_host(self, jobs, sigma_obs: float, K: int, eps: float, obs_op: int = OBS_IDENTITY,
                           stream=None, copy_stream=None, copy_blocks: int = 152, sets: int = 3,
                           out_stream=None):
        """A sequence of analyses whose inputs and results live in page-locked
        host memory (e.g. ``host_empty``), with the copies overlapped: while
        analysis s runs, the inputs of the next analyses are copied in on
        ``copy_stream`` and the results of the previous ones copied out on
        ``out_stream`` (the two directions run side by side).  ``sets``
        device sets of inputs and results rotate; events order every reuse
        (an input set is refilled only after the analysis that read it, a
        result buffer is rewritten only after its copy-out), so copies of up
        to about (sets - 1) analysis times stay hidden.

        jobs: list of dicts with host tensors ``prior`` [n][d], ``y`` [d],
        ``mask`` [d] or None, ``out`` [n][d], and ``seed`` (and ``offset``).
        Everything is enqueued and the call returns; ``stream`` then holds the
        whole sequence (it waits for the last copy-out).  Returns per job the
        CUDA events (copied_in, analysed, copied_out).

        Copies that overlap an analysis go through the copy engines (they
        take no SMs from it); the first copy-in and the last copy-out, which
        nothing overlaps, run as a copy kernel of ``copy_blocks`` blocks on
        the SMs (``copy_sm``) when the host buffer is page-locked and 16-byte
        sized: measured on GB300, copy-engine transfers of 2 GiB slowed to
        100-150 ms on a busy host while the SMs moved the same bytes in
        25-45 ms (10 ms on a quiet host).  Right after other processes on the
        host free much memory, both kinds of copy run far slower for their
        first gigabytes (a 2 GiB copy-out measured 927, 76, then 11 ms)."""
        torch = _torch()
        if not jobs:
            return []
        if sets < 2:
            raise ValueError("analyses_from_host needs at least two device sets")
        s = stream if stream is not None else torch.cuda.current_stream()
        cs = copy_stream if copy_stream is not None else torch.cuda.Stream()
        co = out_stream if out_stream is not None else torch.cuda.Stream()
        p0 = jobs[0]["prior"]
        n, d = p0.shape
        for j in jobs:
            if tuple(j["prior"].shape) != (n, d) or tuple(j["out"].shape) != (n, d) or tuple(j["y"].shape) != (d,):
                raise ValueError("every job needs prior/out [n][d] and y [d] of the same n, d")
            if j["prior"].is_cuda or j["out"].is_cuda:
                raise ValueError("jobs hold host tensors")
        dev = torch.device("cuda", torch.cuda.current_device())
        has_mask = jobs[0].get("mask") is not None
        nsets = min(int(sets), len(jobs))
        devsets = [dict(prior=torch.empty((n, d), dtype=torch.float32, device=dev),
                        y=torch.empty((d,), dtype=torch.float32, device=dev),
                        mask=torch.empty((d,), dtype=torch.uint8, device=dev) if has_mask else None,
                        out=torch.empty((n, d), dtype=torch.float32, device=dev)) for _ in range(nsets)]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in jobs]
        start = torch.cuda.Event()
        start.record(s)
        cs.wait_event(start)
        co.wait_event(start)

        def move(dst, src, sm, stream_):
            host = src if not src.is_cuda else dst
            nbytes = src.numel() * src.element_size()
            if (sm and copy_blocks > 0 and nbytes % 16 == 0 and dst.data_ptr() % 16 == 0
                    and src.data_ptr() % 16 == 0 and host_registered(host)):
                copy_sm(dst, src, copy_blocks, stream=stream_)
            else:
                dst.copy_(src, non_blocking=True)

        issued = [0]  # copy-ins enqueued so far

        def copy_in(i):
            b, j = devsets[i % nsets], jobs[i]
            with torch.cuda.stream(cs):
                if i >= nsets:
                    cs.wait_event(ev[i - nsets][1])   # the analysis that read this set is done
                move(b["prior"], j["prior"], i == 0, cs)
                move(b["y"], j["y"], i == 0, cs)
                if has_mask:
                    move(b["mask"], j["mask"], i == 0, cs)
                ev[i][0].record(cs)
            issued[0] = i + 1

        copy_in(0)
        for i, j in enumerate(jobs):
            b = devsets[i % nsets]
            # the copy-ins the free sets allow, ahead of this analysis
            while issued[0] < len(jobs) and issued[0] <= i + nsets - 1:
                copy_in(issued[0])
            s.wait_event(ev[i][0])
            if i >= nsets:
                s.wait_event(ev[i - nsets][2])    # this result buffer has been copied out
            self.analysis(b["prior"], b["y"], b["mask"], sigma_obs, K, eps, obs_op, seed=j.get("seed", 0),
                          offset=j.get("offset", 0), out=b["out"], stream=s)
            ev[i][1].record(s)
            with torch.cuda.stream(co):
                co.wait_event(ev[i][1])
                move(j["out"], b["out"], i == len(jobs) - 1, co)
                ev[i][2].record(co)
        s.wait_event(ev[-1][2])
        self._pipeline_keep = (devsets, cs, co)   # device buffers live until the streams are done
        return ev

    def analysis_minibatch(self, prior, y, mask, sigma_obs: float, K: int, eps: float, perm, J: int,
                           obs_op: int = OBS_IDENTITY, seed: int = 0, offset: int = 0, out=None, stream=None):
        """Analysis with the mini-batch prior score over windows of J members of
        ``perm`` (device int32 permutation of the members)."""
        torch = _torch()
        _dev(prior, torch.float32, "prior")
        _dev(perm, torch.int32, "perm")
        n, d = prior.shape
        if out is None:
            out = torch.empty_like(prior)
        nz = EnsfNoise(None, int(seed) & (2 ** 64 - 1), int(offset) & 0xFFFFFFFF)
        _check(load().ensf_analysis_minibatch(self._h, prior.data_ptr(), n, d, y.data_ptr(),
                                              mask.data_ptr() if mask is not None else None, int(obs_op),
                                              float(sigma_obs), int(K), float(eps), ctypes.byref(nz),
                                              perm.data_ptr(), int(J), out.data_ptr(), _stream_ptr(stream)),
               "ensf_analysis_minibatch")
        return out

    # ---- d-sharded analysis: this handle runs one slice of the state ----
    def shard(self, prior, y, mask, sigma_obs: float, K: int, eps: float, col0: int, obs_op: int = OBS_IDENTITY,
              seed: int = 0, offset: int = 0, noise=None, out=None):
        """Descriptor of this rank's slice (columns col0 .. col0 + d_local - 1
        of the state) for shard_prep / shard_gram / shard_update; the tensors
        are kept alive in it."""
        torch = _torch()
        _dev(prior, torch.float32, "prior")
        n, d_local = prior.shape
        _dev(y, torch.float32, "y")
        if tuple(y.shape) != (d_local,):
            raise ValueError(f"y must have shape {(d_local,)}")
        if mask is not None:
            _dev(mask, torch.uint8, "mask")
            if tuple(mask.shape) != (d_local,):
                raise ValueError(f"mask must have shape {(d_local,)}")
        if noise is not None:
            _dev(noise, torch.float32, "noise")
            if tuple(noise.shape) != (K + 1, n, d_local):
                raise ValueError(f"noise must have shape {(K + 1, n, d_local)}")
        if out is None:
            out = torch.empty_like(prior)
        _dev(out, torch.float32, "out")
        if tuple(out.shape) != (n, d_local):
            raise ValueError(f"out must have shape {(n, d_local)}")
        desc = EnsfShard(prior.data_ptr(), n, d_local, int(col0), y.data_ptr(),
                         mask.data_ptr() if mask is not None else None, int(obs_op), float(sigma_obs), int(K),
                         float(eps),
                         EnsfNoise(noise.data_ptr() if noise is not None else None, int(seed) & (2 ** 64 - 1),
                                   int(offset) & 0xFFFFFFFF), out.data_ptr())
        desc._keep = (prior, y, mask, noise, out)
        desc.out_tensor = out
        return desc

    def shard_splits(self, n: int, d_local: int) -> int:
        """Split-K partial Grams per step that shard_gram writes for (n, d_local)."""
        S = ctypes.c_int(0)
        _check(load().ensf_shard_splits(self._h, int(n), int(d_local), ctypes.byref(S)), "ensf_shard_splits")
        return int(S.value)

    def shard_prep(self, desc, norms, stream=None):
        """Preparation of this slice; writes its shares of the FP64 norms to ``norms`` [n]."""
        torch = _torch()
        _dev(norms, torch.float64, "norms")
        if norms.numel() != desc.n:
            raise ValueError(f"norms must hold {desc.n} doubles")
        _check(load().ensf_shard_prep(self._h, ctypes.byref(desc), norms.data_ptr(), _stream_ptr(stream)),
               "ensf_shard_prep")

    def shard_gram(self, desc, k: int, partial, stream=None):
        """Step k: this slice's split-K partial Grams into ``partial`` [S][n][n] FP32."""
        torch = _torch()
        _dev(partial, torch.float32, "partial")
        if partial.dim() != 3 or tuple(partial.shape[1:]) != (desc.n, desc.n) or \
                partial.shape[0] != self.shard_splits(desc.n, desc.d_local):
            raise ValueError("partial must be [S][n][n] with S = shard_splits(n, d_local)")
        _check(load().ensf_shard_gram(self._h, ctypes.byref(desc), int(k), partial.data_ptr(), _stream_ptr(stream)),
               "ensf_shard_gram")

    def shard_update(self, desc, k: int, partials, norms, stream=None):
        """Step k: weights from every rank's partials ([R*S][n][n], rank
        order) and the summed norms, then W X + score + update of this slice."""
        torch = _torch()
        _dev(partials, torch.float32, "partials")
        _dev(norms, torch.float64, "norms")
        if partials.dim() != 3 or tuple(partials.shape[1:]) != (desc.n, desc.n) or norms.numel() != desc.n:
            raise ValueError("partials must be [splits][n][n] and norms [n]")
        _check(load().ensf_shard_update(self._h, ctypes.byref(desc), int(k), partials.data_ptr(),
                                        int(partials.shape[0]), norms.data_ptr(), _stream_ptr(stream)),
               "ensf_shard_update")

    def set_tuning(self, n: int, d: int, gram_tile_n: int, gram_stages: int, gram_k_block: int = 64,
                   gram_splits: int = 0, wx_tile_n: int = 0, gram_cta_pair: int = 0, gram_noise_warps: int = 0,
                   gram_fp32_particles: int = 0, noise_inline: int = 0, pdl: int = -1, gram_fused_softmax: int = 0):
        """Record tensor-core launch shapes (and the noise placement,
        ``noise_inline`` 0 = Gram warps, 1 = W X epilogue, 2 = side-stream
        kernel, and whether the step kernels use programmatic dependent
        launch, ``pdl`` 1/0, -1 = keep) for analyses of this (n, d) without
        timing them (e.g. a report saved from ``autotune``)."""
        t = EnsfTuning(gram_tile_n=gram_tile_n, gram_stages=gram_stages, gram_splits=gram_splits,
                       wx_tile_n=wx_tile_n, gram_k_block=gram_k_block, gram_cta_pair=gram_cta_pair,
                       gram_noise_warps=gram_noise_warps, gram_fp32_particles=gram_fp32_particles,
                       noise_inline=noise_inline, pdl=pdl, gram_fused_softmax=gram_fused_softmax)
        _check(load().ensf_set_tuning(self._h, int(n), int(d), ctypes.byref(t)), "ensf_set_tuning")

    def autotune(self, prior, y, mask, sigma_obs: float, eps: float, obs_op: int = OBS_IDENTITY, seed: int = 0,
                 out=None, stream=None) -> dict:
        """Pick the tensor-core launch shapes for this (n, d); overwrites ``out``."""
        torch = _torch()
        _dev(prior, torch.float32, "prior")
        n, d = prior.shape
        if out is None:
            out = torch.empty_like(prior)
        nz = EnsfNoise(None, int(seed) & (2 ** 64 - 1), 0)
        rep = EnsfTuning()
        _check(load().ensf_autotune(self._h, prior.data_ptr(), n, d, y.data_ptr(),
                                    mask.data_ptr() if mask is not None else None, int(obs_op), float(sigma_obs),
                                    float(eps), ctypes.byref(nz), out.data_ptr(), ctypes.byref(rep),
                                    _stream_ptr(stream)), "ensf_autotune")
        return {f: getattr(rep, f) for f, _ in EnsfTuning._fields_}

    def _batch_args(self, filters, outs=None):
        """Instance table, workspace base and size, and the output tensors of
        a batched call (the inputs are kept alive in the returned tuple)."""
        torch = _torch()
        lib = load()
        insts = (EnsfInstance * len(filters))()
        keep = []
        outs = outs or [None] * len(filters)
        results = []
        for i, f in enumerate(filters):
            prior = _dev(f["prior"], torch.float32, "prior")
            y = _dev(f["y"], torch.float32, "y")
            mask = f.get("mask")
            if mask is not None:
                _dev(mask, torch.uint8, "mask")
            out = outs[i] if outs[i] is not None else torch.empty_like(prior)
            n, d = prior.shape
            noise = f.get("noise")
            insts[i] = EnsfInstance(prior.data_ptr(), n, d, y.data_ptr(),
                                    mask.data_ptr() if mask is not None else None, int(f.get("obs_op", 0)),
                                    float(f["sigma_obs"]),
                                    EnsfNoise(noise.data_ptr() if noise is not None else None,
                                              int(f.get("seed", 0)) & (2 ** 64 - 1), int(f.get("offset", 0))),
                                    out.data_ptr())
            keep.append((prior, y, mask, noise))
            results.append(out)
        nbytes = lib.ensf_batch_workspace_bytes(ctypes.byref(self.cfg), insts, len(filters))
        if nbytes == 0:
            raise ValueError("batched analysis needs tensor-core precisions and valid shapes")
        if getattr(self, "_batch_ws", None) is None or self._batch_ws.numel() < nbytes + 256:
            self._batch_ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = (self._batch_ws.data_ptr() + 255) // 256 * 256
        return insts, ctypes.c_void_p(base), nbytes, results, keep

    def analysis_batched(self, filters, K: int, eps: float, outs=None, stream=None):
        """Batched analysis of independent filters.  ``filters`` is a list of
        dicts with device tensors ``prior`` [n][d], ``y`` [d], optional ``mask``
        [d], and ``sigma_obs``, ``obs_op``, ``seed``, ``offset``; returns the
        list of analysis ensembles."""
        insts, base, nbytes, results, _keep = self._batch_args(filters, outs)
        _check(load().ensf_analysis_batched(self._h, insts, len(filters), int(K), float(eps), base, nbytes,
                                            _stream_ptr(stream)), "ensf_analysis_batched")
        return results

    def autotune_batched(self, filters, eps: float, stream=None) -> dict:
        """Pick the k-range per Gram work item of batched analyses of these
        filters (overwrites their outputs); returns the choice and the time
        of its K = 8 trial analysis."""
        insts, base, nbytes, _results, _keep = self._batch_args(filters)
        chunk, ms = ctypes.c_int(0), ctypes.c_float(0.0)
        _check(load().ensf_autotune_batched(self._h, insts, len(filters), float(eps), base, nbytes,
                                            ctypes.byref(chunk), ctypes.byref(ms), _stream_ptr(stream)),
               "ensf_autotune_batched")
        return {"kb_chunk": chunk.value, "trial_ms_k8": ms.value}

    def set_batch_tuning(self, kb_chunk: int) -> None:
        """Record the k-range per batched Gram work item (8, 16, 32 or 64)."""
        _check(load().ensf_set_batch_tuning(self._h, int(kb_chunk)), "ensf_set_batch_tuning")

    def weights(self, z, prior, t: float, eps: float, stream=None):
        """Weights w_ij of Eq. 16 at pseudo-time t; returns [n][n_x] FP32."""
        n, n_x, d = _weights_shapes(z, prior)
        torch = _torch()
        _dev(z, torch.float32, "z")
        _dev(prior, torch.float32, "prior")
        _same_device(z, prior=prior)
        with torch.cuda.device(z.device):
            w = torch.empty((n, n_x), dtype=torch.float32, device=z.device)
            _check(load().ensf_weights(self._h, z.data_ptr(), n, prior.data_ptr(), n_x, d, float(t), float(eps),
                                       w.data_ptr(), _stream_ptr(stream)), "ensf_weights")
        return w

    def profile_enable(self, on: bool = True) -> None:
        _check(load().ensf_profile_enable(self._h, 1 if on else 0), "ensf_profile_enable")

    def profile_read(self) -> dict:
        """{kind: (launches, timed_launches, total_ms)} since the last enable."""
        arr = (EnsfProfileEntry * 16)()
        cnt = ctypes.c_int()
        _check(load().ensf_profile_read(self._h, arr, 16, ctypes.byref(cnt)), "ensf_profile_read")
        return {arr[i].name.decode(): (arr[i].launches, arr[i].timed_launches, arr[i].total_ms)
                for i in range(min(cnt.value, 16))}

    def status_sync(self, stream=None) -> int:
        return int(load().ensf_status_sync(self._h, _stream_ptr(stream)))


def _weights_shapes(z, prior, out=None):
    """(n, n_x, d) of particles z [n][d] against members prior [n_x][d],
    checked before anything reaches the device: the C side sees only
    pointers, so a short prior or a small `out` would be read or written out
    of bounds there."""
    if getattr(z, "dim", None) is None or getattr(prior, "dim", None) is None:
        raise TypeError("z and prior must be tensors")
    if z.dim() != 2 or prior.dim() != 2:
        raise ValueError(f"z and prior must be 2-D, got {tuple(z.shape)} and {tuple(prior.shape)}")
    n, d = z.shape
    n_x = prior.shape[0]
    if prior.shape[1] != d:
        raise ValueError(f"prior has {prior.shape[1]} state entries per member, z has {d}")
    if out is not None:
        if getattr(out, "dim", None) is None or tuple(out.shape) != (n, n_x):
            raise ValueError(f"out must have shape {(n, n_x)}, got {tuple(getattr(out, 'shape', ()))}")
    return int(n), int(n_x), int(d)


def _same_device(ref, **others):
    for name, t in others.items():
        if t is not None and t.device != ref.device:
            raise ValueError(f"{name} is on {t.device}, z on {ref.device}")


HOST_SMALL_PAGES = 1
HOST_ANY_NODE = 2


def host_empty(shape, dtype=None, huge_pages: bool = True, near_device: bool = True):
    """A page-locked host tensor from ensf_host_alloc: backed by huge pages
    (where the kernel offers them) so that copies to and from the device keep
    their speed right after large kernels, and placed on the host NUMA node
    closest to the current device.  Zeroed; freed when the tensor is
    garbage-collected."""
    import weakref

    import numpy as np
    import torch
    dtype = dtype or torch.float32
    shape = tuple(int(v) for v in shape)
    count = 1
    for v in shape:
        count *= v
    itemsize = torch.empty((), dtype=dtype).element_size()
    nbytes = max(count * itemsize, 1)
    lib = load()
    ptr = ctypes.c_void_p()
    flags = (0 if huge_pages else HOST_SMALL_PAGES) | (0 if near_device else HOST_ANY_NODE)
    _check(lib.ensf_host_alloc(nbytes, flags, ctypes.byref(ptr)), "ensf_host_alloc")
    raw = (ctypes.c_uint8 * nbytes).from_address(ptr.value)
    t = torch.from_numpy(np.ctypeslib.as_array(raw)).view(dtype)[:count].view(shape)
    weakref.finalize(t, lib.ensf_host_free, ctypes.c_void_p(ptr.value))
    return t


def copy_sm(dst, src, blocks: int = 152, stream=None):
    """dst.copy_(src) by a copy kernel on the SMs (ensf_copy_sm): either
    tensor may live in device memory or in page-locked host memory."""
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nbytes or not dst.is_contiguous() or not src.is_contiguous():
        raise ValueError("copy_sm: contiguous tensors of equal byte size")
    _check(load().ensf_copy_sm(dst.data_ptr(), src.data_ptr(), nbytes, int(blocks), _stream_ptr(stream)),
           "ensf_copy_sm")
    return dst


def host_registered(t) -> bool:
    """Whether a host tensor's memory is page-locked with the CUDA driver."""
    r = ctypes.c_int(0)
    _check(load().ensf_host_registered(t.data_ptr(), ctypes.byref(r)), "ensf_host_registered")
    return bool(r.value)


def host_huge_fraction(t) -> float:
    """Share of a host tensor's bytes backed by huge pages right now."""
    frac = ctypes.c_double(0.0)
    _check(load().ensf_host_huge_fraction(t.data_ptr(), t.numel() * t.element_size(), ctypes.byref(frac)),
           "ensf_host_huge_fraction")
    return float(frac.value)


def host_numa(t):
    """(NUMA node of the page holding the tensor's first byte, host node
    closest to the current device); -1 where unknown."""
    node, dev_node = ctypes.c_int(-1), ctypes.c_int(-1)
    _check(load().ensf_host_numa(t.data_ptr(), ctypes.byref(node), ctypes.byref(dev_node)), "ensf_host_numa")
    return int(node.value), int(dev_node.value)


def weights_static(z, prior, t: float, eps: float, out=None, stream=None):
    """Weights of Eq. 16 (FP32 Gram on centred operands) through the
    allocation-free entry point: no handle, no workspace; at most 256
    particles, 256 members and 524288 state entries.  Runs on z's device."""
    n, n_x, d = _weights_shapes(z, prior, out)
    torch = _torch()
    _dev(z, torch.float32, "z")
    _dev(prior, torch.float32, "prior")
    if out is not None:
        _dev(out, torch.float32, "out")
    _same_device(z, prior=prior, out=out)
    with torch.cuda.device(z.device):
        w = out if out is not None else torch.empty((n, n_x), dtype=torch.float32, device=z.device)
        _check(load().ensf_weights_static(z.data_ptr(), n, prior.data_ptr(), n_x, d, float(t), float(eps),
                                          w.data_ptr(), _stream_ptr(stream)), "ensf_weights_static")
    return w


class SQG:
    """GPU two-level SQG integrator over a batch of members (theta [B][2][n][n])."""

    def __init__(self, batch: int, n: int = 128, L: float = 20.0, H: float = 1.0, N_over_f: float = 1.0,
                 shear: float = 1.0, dt: float = 0.025, tau_diss: float = 0.1, diffusion: bool = True,
                 tau_relax: float = 0.0):
        torch = _torch()
        lib = load()
        self.params = EnsfSqgParams(int(n), float(L), float(H), float(N_over_f), float(shear), float(dt),
                                    float(tau_diss), 1 if diffusion else 0, float(tau_relax))
        nbytes = lib.ensf_sqg_workspace_bytes(ctypes.byref(self.params), int(batch))
        if nbytes == 0:
            raise ValueError("invalid SQG parameters")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(lib.ensf_sqg_create(ctypes.byref(self.params), int(batch), ctypes.c_void_p(base), nbytes,
                                   ctypes.byref(h)), "ensf_sqg_create")
        self._h = h
        self.batch, self.n = int(batch), int(n)

    def run(self, theta, nsteps: int, stream=None):
        """Advance theta [batch][2][n][n] (CUDA float32, in place) by nsteps RK4 steps."""
        torch = _torch()
        _dev(theta, torch.float32, "theta")
        if tuple(theta.shape) != (self.batch, 2, self.n, self.n):
            raise ValueError(f"theta must be {(self.batch, 2, self.n, self.n)}")
        _check(load().ensf_sqg_run(self._h, theta.data_ptr(), int(nsteps), _stream_ptr(stream)), "ensf_sqg_run")
        return theta

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None and self._h.value:
                load().ensf_sqg_destroy(self._h)
                self._h = None
        except Exception:
            pass


class UNet:
    """The BF16 conv U-Net forecast surrogate (x_{t+Delta} = x_t + net(x_t))."""

    def __init__(self, widths=(32, 64, 128, 256), height: int = 128, width: int = 128, max_batch: int = 16):
        torch = _torch()
        lib = load()
        self.cfg = EnsfUnetConfig(2, 2, (ctypes.c_int * 4)(*[int(w) for w in widths]), int(height), int(width),
                                  int(max_batch))
        self.nparams = int(lib.ensf_unet_param_count(ctypes.byref(self.cfg)))
        nbytes = lib.ensf_unet_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0 or self.nparams == 0:
            raise ValueError("invalid U-Net configuration")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(lib.ensf_unet_create(ctypes.byref(self.cfg), ctypes.c_void_p(base), nbytes, ctypes.byref(h)),
               "ensf_unet_create")
        self._h = h
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device="cuda")

    def set_params(self, params, stream=None):
        torch = _torch()
        _dev(params, torch.float32, "params")
        if params.numel() != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters")
        _check(load().ensf_unet_set_params(self._h, params.data_ptr(), _stream_ptr(stream)), "ensf_unet_set_params")

    def get_params(self, stream=None):
        torch = _torch()
        out = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        _check(load().ensf_unet_get_params(self._h, out.data_ptr(), _stream_ptr(stream)), "ensf_unet_get_params")
        return out

    def get_moments(self, stream=None):
        """AdamW state: (first moments, second moments, steps since set_params)."""
        torch = _torch()
        m = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        v = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        step = ctypes.c_int64(0)
        _check(load().ensf_unet_get_moments(self._h, m.data_ptr(), v.data_ptr(), ctypes.byref(step),
                                            _stream_ptr(stream)), "ensf_unet_get_moments")
        return m, v, int(step.value)

    def forward(self, x, stream=None):
        torch = _torch()
        _dev(x, torch.float32, "x")
        y = torch.empty_like(x)
        _check(load().ensf_unet_forward(self._h, x.data_ptr(), x.shape[0], y.data_ptr(), _stream_ptr(stream)),
               "ensf_unet_forward")
        return y

    def gradients(self, x, target, stream=None):
        torch = _torch()
        g = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        _check(load().ensf_unet_gradients(self._h, x.data_ptr(), target.data_ptr(), x.shape[0], g.data_ptr(),
                                          self.loss_buf.data_ptr(), _stream_ptr(stream)), "ensf_unet_gradients")
        return g, self.loss_buf

    def train_step(self, x, target, lr: float, weight_decay: float = 0.0, stream=None):
        """One AdamW step; returns the device loss scalar (before the step)."""
        _check(load().ensf_unet_train_step(self._h, x.data_ptr(), target.data_ptr(), x.shape[0], float(lr),
                                           float(weight_decay), self.loss_buf.data_ptr(), _stream_ptr(stream)),
               "ensf_unet_train_step")
        return self.loss_buf

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None and self._h.value:
                load().ensf_unet_destroy(self._h)
                self._h = None
        except Exception:
            pass


def philox_normal(seed: int, offset: int, k0: int, count: int, n: int, d: int, stream=None):
    torch = _torch()
    out = torch.empty((count, n, d), dtype=torch.float32, device="cuda")
    _check(load().ensf_philox_normal(int(seed) & (2 ** 64 - 1), int(offset), int(k0), int(count), int(n), int(d),
                                     out.data_ptr(), _stream_ptr(stream)), "ensf_philox_normal")
    return out


def row_norms(x, stream=None):
    torch = _torch()
    _dev(x, torch.float32, "x")
    out = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
    _check(load().ensf_row_norms(x.data_ptr(), x.shape[0], x.shape[1], out.data_ptr(), _stream_ptr(stream)),
           "ensf_row_norms")
    return out


def relax_spread(prior, z, factor: float = 1.0, mode: str = "spread", stream=None):
    """Relax the analysis z [n][d] toward the prior, in place: ``mode`` "spread"
    rescales the anomalies to the prior spread, "perturbations" blends them
    with the prior anomalies."""
    torch = _torch()
    _dev(prior, torch.float32, "prior")
    _dev(z, torch.float32, "z")
    n, d = z.shape
    _check(load().ensf_relax_spread(prior.data_ptr(), z.data_ptr(), n, d, float(factor),
                                    {"spread": 0, "perturbations": 1}[mode], _stream_ptr(stream)),
           "ensf_relax_spread")
    return z


def selftest_timeouts(stream=None):
    """Run the library's two bounded-wait self-tests (an mbarrier that never
    completes, a grid barrier that one block skips); returns the two status
    words, both ETIMEOUT when detection works.  Takes about 4 s."""
    torch = _torch()
    words = torch.zeros(4, dtype=torch.int32, device="cuda")
    _check(load().ensf_selftest_timeouts(words.data_ptr(), _stream_ptr(stream)), "ensf_selftest_timeouts")
    torch.cuda.synchronize()
    return [int(v) for v in words[:2].cpu()]


def model_error(state, coef, seed: int, cycle: int, stream=None):
    """Add the imperfect-model error sum_p coef[p] xi_p to ``state`` [B][d]
    (or [d]) in place; xi_p the counter-based normals at (seed, cycle, p)."""
    torch = _torch()
    _dev(state, torch.float32, "state")
    B, d = (1, state.shape[0]) if state.dim() == 1 else (state.shape[0], state[0].numel())
    c = (ctypes.c_float * len(coef))(*[float(v) for v in coef])
    _check(load().ensf_model_error(state.data_ptr(), B, d, c, len(coef), int(seed) & (2 ** 64 - 1),
                                   int(cycle) & 0xFFFFFFFF, _stream_ptr(stream)), "ensf_model_error")
    return state


def ensemble_stats(z, truth: Optional[object] = None, stream=None):
    """FP64 ensemble mean [d] and, with ``truth``, the RMSE of the mean."""
    torch = _torch()
    _dev(z, torch.float32, "z")
    n, d = z.shape
    lib = load()
    scratch = torch.empty(lib.ensf_stats_scratch_bytes(d) // 8 + 1, dtype=torch.float64, device=z.device)
    mean = torch.empty(d, dtype=torch.float64, device=z.device)
    rmse = torch.empty(1, dtype=torch.float64, device=z.device)
    if truth is not None:
        _dev(truth, torch.float32, "truth")
    _check(lib.ensf_ensemble_stats(z.data_ptr(), n, d, truth.data_ptr() if truth is not None else None,
                                   mean.data_ptr(), rmse.data_ptr() if truth is not None else None,
                                   scratch.data_ptr(), _stream_ptr(stream)), "ensf_ensemble_stats")
    return mean, (rmse if truth is not None else None)


# (gram, wx, tolerance) combinations exercised by the package smoke check
SMOKE_PATHS = [("fp32", "fp32", 1e-4), ("split", "split", 1e-4), ("split", "bf16", 1e-2)]
