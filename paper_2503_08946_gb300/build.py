"""Build the race-checker library ``_build/librc.so`` in-tree for sm_103a.

Each CUDA translation unit is compiled by nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``), the host lowering by g++, and the
objects are linked into one shared library with the static CUDA runtime.
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
LIB = os.path.join(BUILD, "librc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
CUDA_INCLUDE = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

CUDA_SOURCES = ["expand.cu", "sort.cu", "histogram.cu", "scan.cu", "bucket.cu", "runtime.cu", "sort_static.cu", "hash.cu",
                "batch.cu"]
HOST_SOURCES = ["lower.cpp", "jit.cpp", "server.cpp"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + CSRC, "-I" + INCLUDE] + GENCODE


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the race checker")


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "rc.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + list(extra_flags or [])
    jobs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        jobs.append([nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + flags)
    for src in HOST_SOURCES:
        obj = os.path.join(BUILD, src.replace(".cpp", ".o"))
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I" + CSRC, "-I" + INCLUDE, "-I" + CUDA_INCLUDE, "-c",
                     os.path.join(CSRC, src), "-o", obj])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or p.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {cmd[2] if cmd[1] == '-c' else cmd}")
        return p.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in CUDA_SOURCES] + \
           [os.path.join(BUILD, s.replace(".cpp", ".o")) for s in HOST_SOURCES]
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, "-shared", "-o", tmp] + objs + GENCODE + ["-cudart", "static", "-ldl", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
