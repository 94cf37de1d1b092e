"""In-tree build of the EnSF CUDA library (``_lib/libensf.so``) for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically.  No torch types cross
the boundary; the Python binding loads the library with ctypes.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libensf.so")
SOURCES = ["ensf_api.cu", "ensf_simt.cu", "ensf_tc.cu", "ensf_conv.cu", "ensf_static.cu", "ensf_sqg.cu",
           "ensf_unet.cu", "ensf_small.cu", "ensf_host.cu"]
HEADERS = ["ensf_device.cuh", "ensf_internal.h", "ensf_tc.h", "ensf_ptx.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"),
                 shutil.which("nvcc") or ""):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the EnSF CUDA library cannot be built")


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "ensf.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(src: str, obj: str, extra) -> None:
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr",
           "-I", os.path.join(ROOT, "include"), *extra, "-c", src, "-o", obj]
    subprocess.check_call(cmd)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    objs = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as pool:
        futs = []
        for s in SOURCES:
            obj = os.path.join(OUT_DIR, s.replace(".cu", ".o"))
            objs.append(obj)
            futs.append(pool.submit(_compile, os.path.join(CSRC, s), obj, extra))
        for f in futs:
            f.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs,
                           "-L" + cuda_lib, "-lcufft", "-Xlinker", "-rpath", "-Xlinker", cuda_lib])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas-v" in sys.argv))
