"""Build the test-only probe library libnef_probe.so (tests only).

It holds the tensor-core layout probe (k_tc_probe.cu, on the fused pass's own
PTX wrappers and descriptors from csrc/k_view_tc.cuh) and the fold-in encoder's
GEMM on its own (the product kernel csrc/k_gemm_tc.cu plus the nef_tc_gemm
wrapper), for sm_103a.  The product library does not contain these entry points.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2602_02759_gb300", "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnef_probe.so")
SRCS = [os.path.join(HERE, "k_tc_probe.cu"), os.path.join(HERE, "gemm_probe.cu"), os.path.join(CSRC, "k_gemm_tc.cu")]
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "--expt-relaxed-constexpr", "-I", HERE, "-I", CSRC, "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in ("/usr/local/cuda/bin/nvcc", "nvcc"):
        if os.path.sep not in c or os.path.exists(c):
            return c
    return "nvcc"


def build() -> str:
    os.makedirs(OUT, exist_ok=True)
    deps = SRCS + [os.path.join(HERE, "nef_probe.h")] + \
        [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
        return LIB

    def comp(src):
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        r = subprocess.run([_nvcc(), *FLAGS, "-c", src, "-o", obj], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SRCS)) as ex:
        objs = list(ex.map(comp, SRCS))
    r = subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", LIB + ".tmp", *objs,
                        "-cudart", "static", "-Xlinker", "-Bsymbolic"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def load():
    """Load the probe library with its argument types (builds it first if needed)."""
    import ctypes
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.nef_tc_probe.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.nef_tc_probe.restype = ctypes.c_int
        lib.nef_tc_gemm.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, vp, vp]
        lib.nef_tc_gemm.restype = ctypes.c_int
        lib.nef_tc_gemm_split.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int64, vp, vp]
        lib.nef_tc_gemm_split.restype = ctypes.c_int
        _lib = lib
    return _lib


if __name__ == "__main__":
    print(build())
