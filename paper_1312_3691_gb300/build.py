"""Builds libtpmc.so in-tree: CUDA kernels for sm_103a plus the C++ host runtime.

nvcc compiles kernels.cu for sm_103a only; g++ compiles the host sources; the
translation units build in parallel and nvcc links the shared library (CUDA
runtime linked statically).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtpmc.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels.cu", "noalloc.cu", "ceilings.cu"]
CPP_SOURCES = ["api.cpp", "bvh.cpp", "serve.cpp", "tune.cpp"]
HEADERS = ["tpmc_internal.h", "runtime.h", os.path.join("..", "..", "include", "tpmc.h")]
# kernels.cu: float division and square root by the hardware approximations
# (within two units in the last place) instead of the correctly rounded
# sequences, which cost 7-10 % of the trace kernel's throughput in the seeding
# and re-emission arithmetic.  Double precision is unaffected, and so are the
# explicitly rounded intrinsics the watertight triangle test uses.
CU_FLAGS = {"kernels.cu": ["-prec-div=false", "-prec-sqrt=false"]}


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    deps = [path, os.path.abspath(__file__)] + [os.path.join(CSRC, h) for h in HEADERS]
    if os.path.exists(obj) and os.path.getmtime(obj) >= _newest(deps):
        return obj
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", *CU_FLAGS.get(src, []), "-Xcompiler", "-fPIC", "-c",
               path, "-o", obj]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", os.path.join(CUDA_HOME, "include"), "-c", path,
               "-o", obj]
    subprocess.check_call(cmd)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    if shutil.which(NVCC) is None and not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=len(CU_SOURCES) + len(CPP_SOURCES)) as ex:
        objs = list(ex.map(_compile, CU_SOURCES + CPP_SOURCES))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
