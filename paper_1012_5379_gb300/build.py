"""Build libhelm.so in-tree: nvcc for the sm_103a kernels, g++ for the host engine,
translation units compiled in parallel.  Usage: python -m paper_1012_5379_gb300.build"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhelm.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["vcycle_c64.cu", "vcycle_c128.cu", "outer.cu", "convert.cu", "noalloc.cu"]
CPP = ["engine.cpp", "geometry.cpp", "capi.cpp", "profiler.cpp", "serve.cpp", "tma.cpp", "tune.cpp", "autotune.cpp"]
HEADERS = ["poly.h", "helm_internal.h", "device_common.cuh", "vcycle.cuh", "tiles.cuh", "vcycle_launch.cuh", "engine.h", "geometry.h",
           "profiler.h"]


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in CU + CPP + HEADERS]
    files.append(os.path.join(PKG, "..", "include", "helm.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit and link libhelm.so; returns the library path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + os.path.join(CUDA_HOME, "include")]
    jobs = []
    for f in CU:
        jobs.append([NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-c", os.path.join(CSRC, f), "-o", os.path.join(BUILD, f + ".o")])
    cxx = shutil.which("g++") or "g++"
    for f in CPP:
        jobs.append([cxx, "-std=c++17", "-O2", "-fPIC", *inc, "-c", os.path.join(CSRC, f),
                     "-o", os.path.join(BUILD, f + ".o")])
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD, f + ".o") for f in CU + CPP]
    tmp = LIB + ".tmp"
    _run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
