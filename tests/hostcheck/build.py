"""Build the host test double: the product's plan.cpp, batched.cpp and foldin.cpp
compiled with g++ against a fake CUDA runtime and plain-loop launchers (tests only)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2602_02759_gb300", "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnef_hostcheck.so")


def build():
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(CSRC, "plan.cpp"), os.path.join(CSRC, "batched.cpp"), os.path.join(CSRC, "foldin.cpp"),
            os.path.join(HERE, "mock_launchers.cpp"), os.path.join(HERE, "mock_batched.cpp"),
            os.path.join(HERE, "mock_foldin.cpp")]
    deps = srcs + [os.path.join(CSRC, f) for f in ("nef_internal.h", "nef_device.cuh", "nef_batched.h")] + \
        [os.path.join(ROOT, "include", "nef.h")] + \
        [os.path.join(HERE, "shim", f) for f in ("cuda_runtime.h", "cuda.h")]
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
        return LIB
    cmd = ["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I", os.path.join(HERE, "shim"),
           "-I", CSRC, "-I", os.path.join(ROOT, "include"), *srcs, "-o", LIB + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build())
