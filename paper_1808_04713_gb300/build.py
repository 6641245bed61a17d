"""In-tree build of the native library libddh.so (host C++ setup + sm_103a CUDA kernels).

Host sources compile with g++ -O3 (no architecture-specific flags, so the same code builds
on x86-64 and aarch64); CUDA sources with nvcc for sm_103a only.  Objects go to _build/,
the shared library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libddh.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CPP_SRCS = ["ddh_tables.cpp", "ddh_mesh.cpp", "ddh_factor.cpp", "ddh_coarse.cpp"]
CU_SRCS = ["ddh_k_fdm_pass1_f64.cu", "ddh_k_fdm_pass1_f32.cu", "ddh_k_fdm_pass2_f64.cu", "ddh_k_fdm_pass2_f32.cu",
           "ddh_k_edge.cu", "ddh_k_tc.cu", "ddh_k_coarse.cu", "ddh_k_krylov.cu", "ddh_k_misc.cu", "ddh_api.cu",
           "ddh_noalloc.cu"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "ddh.h"))
    jobs = []
    for f in CPP_SRCS:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-variable", "-c", src, "-o", obj]
        jobs.append((obj, [src] + headers, cmd))
    for f in CU_SRCS:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        cmd = [NVCC] + ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
        jobs.append((obj, [src] + headers, cmd))
    todo = [j for j in jobs if force or _stale(j[0], j[1])]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 4))) as ex:
        for out in ex.map(lambda j: _run(j[2]), todo):
            if verbose and out.strip():
                print(out)
    objs = [j[0] for j in jobs]
    if force or todo or not os.path.exists(LIB):
        _run([NVCC] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart", "-lpthread"])
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
