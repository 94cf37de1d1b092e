"""The allocation-free weights entry point, ensf_weights_static.

Some callers cannot allocate device memory: applications whose own pool owns
every device allocation, and loops that must never reach an allocation that
could synchronise the device.  ensf_weights_static serves them with a static
device scratch array instead of a caller workspace.  This test calls it
through the C ABI several times in a row -- the largest case first, so that
the later, smaller calls run over whatever the earlier ones left in the shared
array -- and checks every result against the FP64 oracle's weights (Eq. 16)
at the tolerance of the weights parity test, and against the workspace-based
ensf_weights.  One case sits at a small pseudo-time with a forecast ensemble
far from zero mean, where the expanded log-kernel would lose its accuracy
without centring.  It lives in its own file so that it runs last; it passes
alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as o

pytestmark = pytest.mark.gpu

WEIGHT_ATOL = 2e-4  # as in test_gpu_parity.test_weights_match_oracle
MIN_GAP = 1e-2      # rows whose top-two log-kernels lie closer count as tied there too


def _case(seed, n, n_x, d, t, offset=0.2, spread=0.5, mix=False):
    g = np.random.default_rng(seed)
    X = (g.standard_normal((n_x, d)) * spread + offset).astype(np.float32)
    alpha = 1.0 - t * 0.95
    if mix:
        # particles between two members, so that the weights are spread
        a, b = g.integers(0, n_x, n), g.integers(0, n_x, n)
        lam = g.uniform(0.3, 0.7, (n, 1))
        base = lam * X[a] + (1.0 - lam) * X[b]
    else:
        base = X[g.integers(0, n_x, n)]
    Z = (alpha * base + np.sqrt(t) * 0.05 * spread * g.standard_normal((n, d))).astype(np.float32)
    return Z, X


# largest first: each later call reads the static array over an earlier call's leftovers
CASES = [
    # (seed, n, n_x, d, t, offset, spread, mix)
    (32, 200, 256, 20480, 0.3, 0.2, 0.5, False),
    (33, 64, 64, 8192, 0.05, 1.0, 0.01, True),   # small t, mean far from zero
    (31, 37, 45, 4104, 0.6, 0.2, 0.5, False),
]


def _static(lib, z, n, x, n_x, d, t, w, stream):
    return lib.ensf_weights_static(ctypes.c_void_p(z.data_ptr()), n, ctypes.c_void_p(x.data_ptr()), n_x, d,
                                   ctypes.c_float(t), ctypes.c_float(0.05), ctypes.c_void_p(w.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))


def test_weights_static_matches_oracle_over_leftovers():
    import torch
    from paper_2407_12168_gb300 import ensf

    lib = ensf.load()
    stream = torch.cuda.current_stream()
    spread_rows = 0
    for seed, n, n_x, d, t, offset, spread, mix in CASES:
        Z, X = _case(seed, n, n_x, d, t, offset, spread, mix)
        z = torch.from_numpy(Z).cuda()
        x = torch.from_numpy(X).cuda()
        w = torch.full((n, n_x), float("nan"), dtype=torch.float32, device="cuda")
        st = _static(lib, z, n, x, n_x, d, t, w, stream)
        assert st == ensf.OK, lib.ensf_last_error().decode()
        ws = ensf.Filter(max(n, n_x), d, gram="fp32", wx="fp32").weights(z, x, t, 0.05)
        torch.cuda.synchronize()
        got, via_ws = w.cpu().numpy(), ws.cpu().numpy()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got.sum(axis=1), 1.0, atol=1e-5)
        s = o.schedule(t, 0.05)
        for i in range(n):
            ref, logit = o.weights(X, Z[i], s["alpha"], s["beta2"])
            top = np.sort(logit)
            if n_x > 1 and top[-1] - top[-2] <= MIN_GAP:
                continue
            np.testing.assert_allclose(got[i], ref, atol=WEIGHT_ATOL, err_msg=f"case seed {seed}, row {i}")
            np.testing.assert_allclose(via_ws[i], ref, atol=WEIGHT_ATOL)
            spread_rows += int(ref.max() < 0.99)
    # the small-t case really exercises the softmax (weights not one-hot)
    assert spread_rows >= 32


def test_weights_static_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2407_12168_gb300 import ensf

    lib = ensf.load()
    z = torch.zeros((257, 64), device="cuda")
    x = torch.zeros((8, 64), device="cuda")
    w = torch.zeros((257, 8), device="cuda")
    stream = torch.cuda.current_stream()
    assert _static(lib, z, 257, x, 8, 64, 0.5, w, stream) == ensf.EINVAL
    assert b"256" in lib.ensf_last_error()
    # a state longer than the static centre holds is refused before any launch
    assert _static(lib, z, 8, x, 8, 524288 + 8, 0.5, w, stream) == ensf.EINVAL
    assert b"524288" in lib.ensf_last_error()
