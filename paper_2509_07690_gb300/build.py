"""Build libhylu.so in-tree for sm_103a: host preprocessing (g++) and the CUDA
kernels + C ABI (nvcc), compiled in parallel and linked into one shared
library next to this file.  No CMake."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "libhylu.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SRCS = ["host/mwm.cpp", "host/amd.cpp", "host/nd.cpp", "host/symbolic.cpp", "host/analyze.cpp",
             "host/batch.cpp", "host/serialize.cpp", "host/gemm_plan.cpp",
             "host/seq_segments.cpp"]
CUDA_SRCS = ["kernels.cu", "capi.cu", "peak.cu", "static_solve.cu", "tc_gemm.cu"]


def _sources():
    out = []
    for root, _, files in os.walk(CSRC):
        for f in files:
            out.append(os.path.join(root, f))
    out.append(os.path.join(os.path.dirname(HERE), "include", "hylu.h"))
    return out


def _stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(p) > t for p in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return SO
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    objs = []
    for src in HOST_SRCS:
        o = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-c", os.path.join(CSRC, src), "-o", o])
    for src in CUDA_SRCS:
        o = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(o)
        jobs.append([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-c", os.path.join(CSRC, src), "-o", o])
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        for r in ex.map(_run, jobs):
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
    tmp = SO + f".tmp{os.getpid()}"
    # -ldl: the NVTX ranges look up a profiler's injection library with dlopen
    # (part of libc from glibc 2.34 on, of libdl before)
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"])
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
