"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point that include/ensf.h declares, and rejects bad arguments on
the host before touching a device.  No compute call runs here."""
import ctypes
import os
import re

import pytest

from paper_2407_12168_gb300 import ensf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ensf_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = ensf.load()
    declared = _declared_symbols()
    assert len(declared) >= 12
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert ensf.library_path().endswith("libensf.so")


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in ensf._SIGNATURES}
    assert _declared_symbols() <= bound


def test_workspace_size_rules():
    lib = ensf.load()
    good = ensf.EnsfConfig(20, 8192, ensf.PREC_FP32, ensf.PREC_FP32, 0)
    assert lib.ensf_workspace_bytes(ctypes.byref(good)) > 20 * 20 * 4
    for bad in [ensf.EnsfConfig(0, 8192, 0, 0, 0), ensf.EnsfConfig(20, 8190, 0, 0, 0),
                ensf.EnsfConfig(20, 8192, 7, 0, 0), ensf.EnsfConfig(9000, 8192, 0, 0, 0)]:
        assert lib.ensf_workspace_bytes(ctypes.byref(bad)) == 0
    assert lib.ensf_workspace_bytes(None) == 0
    split = ensf.EnsfConfig(1024, 524288, ensf.PREC_SPLIT_BF16X3, ensf.PREC_BF16, 0)
    plain = ensf.EnsfConfig(1024, 524288, ensf.PREC_FP32, ensf.PREC_FP32, 0)
    # split planes: X hi/lo, Z hi/lo (4 x 1 GiB) and X^T hi (1 GiB)
    assert lib.ensf_workspace_bytes(ctypes.byref(split)) - lib.ensf_workspace_bytes(ctypes.byref(plain)) \
        >= 5 * 1024 * 524288 * 2


def test_host_argument_errors_need_no_device():
    lib = ensf.load()
    cfg = ensf.EnsfConfig(20, 8192, 0, 0, 0)
    h = ctypes.c_void_p()
    assert lib.ensf_create(ctypes.byref(cfg), None, 1 << 20, ctypes.byref(h)) == ensf.EINVAL
    assert lib.ensf_create(ctypes.byref(cfg), ctypes.c_void_p(0x1001), 1 << 30, ctypes.byref(h)) == ensf.EINVAL
    assert lib.ensf_create(ctypes.byref(cfg), ctypes.c_void_p(0x1000), 1 << 30, None) == ensf.EINVAL
    assert lib.ensf_create(ctypes.byref(cfg), ctypes.c_void_p(0x1000), 16, ctypes.byref(h)) == ensf.ENOMEM
    assert b"workspace" in lib.ensf_last_error()
    noise = ensf.EnsfNoise(None, 1, 0)
    assert lib.ensf_analysis(None, 0x1000, 4, 8, 0x1000, None, 0, 1.0, 3, 0.05, ctypes.byref(noise),
                             0x2000, None) == ensf.EINVAL
    assert lib.ensf_status_sync(None, None) == ensf.EINVAL
    assert lib.ensf_destroy(None) == ensf.EINVAL
    assert lib.ensf_philox_normal(1, 0, 0, 1, 1, 6, 0x1000, None) == ensf.EINVAL
    assert lib.ensf_row_norms(None, 1, 8, 0x1000, None) == ensf.EINVAL
    for s in range(7):
        assert lib.ensf_status_string(s).startswith(b"ENSF_")


def test_binding_fails_loudly_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError):
        ensf.Filter(4, 64)


def test_weights_wrappers_reject_mismatched_shapes_on_the_host():
    """The weights wrappers check shapes before anything reaches the device:
    the C side sees only pointers, so a prior with fewer columns than z, or
    an `out` of the wrong shape, would be read or written out of bounds."""
    import torch
    z = torch.zeros((4, 16))
    with pytest.raises(ValueError, match="state entries"):
        ensf.weights_static(z, torch.zeros((3, 8)), 0.5, 0.05)
    with pytest.raises(ValueError, match="2-D"):
        ensf.weights_static(z, torch.zeros((3, 16, 1)), 0.5, 0.05)
    with pytest.raises(ValueError, match="2-D"):
        ensf.weights_static(torch.zeros(16), torch.zeros((3, 16)), 0.5, 0.05)
    with pytest.raises(ValueError, match="out must have shape"):
        ensf.weights_static(z, torch.zeros((3, 16)), 0.5, 0.05, out=torch.zeros((4, 2)))
    with pytest.raises(ValueError, match="state entries"):
        ensf._weights_shapes(z, torch.zeros((3, 32)))
    assert ensf._weights_shapes(z, torch.zeros((3, 16)), torch.zeros((4, 3))) == (4, 3, 16)
