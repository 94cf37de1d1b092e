"""The allocation-free weights entry point, ensf_weights_static.

Some callers cannot allocate device memory: applications whose own pool owns
every device allocation, and loops that must never reach an allocation that
could synchronise the device.  ensf_weights_static serves them with a static
device scratch array instead of a caller workspace.  This test calls it
through the C ABI twice in a row (different shapes, so the second call runs
over whatever the first left in the shared array) and checks each result
against the workspace-based ensf_weights with the FP32 Gram, to the same
tolerance as the weights parity test.  It lives in its own file so that it
runs last; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WEIGHT_ATOL = 2e-4  # as in test_gpu_parity.test_weights_match_oracle


def _case(seed, n, n_x, d, t):
    g = np.random.default_rng(seed)
    X = (g.standard_normal((n_x, d)) * 0.5 + 0.2).astype(np.float32)
    alpha = 1.0 - t * 0.95
    Z = (alpha * X[g.integers(0, n_x, n)] + np.sqrt(t) * 0.05 * g.standard_normal((n, d))).astype(np.float32)
    return Z, X


def test_weights_static_matches_workspace_entry_point():
    import torch
    from paper_2407_12168_gb300 import ensf

    lib = ensf.load()
    stream = torch.cuda.current_stream()
    cases = [(31, 37, 45, 4104, 0.6), (32, 200, 256, 2056, 0.3)]
    for seed, n, n_x, d, t in cases:
        Z, X = _case(seed, n, n_x, d, t)
        z = torch.from_numpy(Z).cuda()
        x = torch.from_numpy(X).cuda()
        w = torch.full((n, n_x), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.ensf_weights_static(ctypes.c_void_p(z.data_ptr()), n, ctypes.c_void_p(x.data_ptr()), n_x, d,
                                     ctypes.c_float(t), ctypes.c_float(0.05), ctypes.c_void_p(w.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert st == ensf.OK, lib.ensf_last_error().decode()
        ref = ensf.Filter(max(n, n_x), d, gram="fp32", wx="fp32").weights(z, x, t, 0.05)
        torch.cuda.synchronize()
        got, want = w.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got.sum(axis=1), 1.0, atol=1e-5)
        np.testing.assert_allclose(got, want, atol=WEIGHT_ATOL)


def test_weights_static_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2407_12168_gb300 import ensf

    lib = ensf.load()
    z = torch.zeros((257, 64), device="cuda")
    x = torch.zeros((8, 64), device="cuda")
    w = torch.zeros((257, 8), device="cuda")
    st = lib.ensf_weights_static(ctypes.c_void_p(z.data_ptr()), 257, ctypes.c_void_p(x.data_ptr()), 8, 64,
                                 ctypes.c_float(0.5), ctypes.c_float(0.05), ctypes.c_void_p(w.data_ptr()), None)
    assert st == ensf.EINVAL
    assert b"256" in lib.ensf_last_error()
