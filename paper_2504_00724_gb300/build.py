"""Build libccm.so in-tree: host setup (C++17) and CUDA kernels for sm_103a.

Translation units are compiled in parallel and linked with nvcc; the result lands next to
this file.  Re-running skips the build when no source is newer than the library.  Host code
is compiled with floating-point contraction off, so that the setup (whose discrete choices,
such as whether the boundary crosses a cell edge or only touches a grid vertex, can hang on
the last bit) gives the same result on x86-64 and on AArch64, where GCC would otherwise fuse
multiply-adds.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libccm.so")
BUILD = os.path.join(HERE, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CXX_SOURCES = ["geometry.cpp", "discretize.cpp", "hierarchy.cpp", "host_api.cpp"]
CU_SOURCES = ["solver.cu", "fitdev.cu"]


def _sources():
    out = [os.path.join(CSRC, f) for f in CXX_SOURCES + CU_SOURCES]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    out.append(os.path.join(INCLUDE, "ccm.h"))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for f in CXX_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        jobs.append(["g++", "-std=c++17", "-O3", "-ffp-contract=off", "-fPIC", "-Wall", "-I", INCLUDE, "-c",
                     os.path.join(CSRC, f), "-o", o])
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        jobs.append([NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", INCLUDE, "-c", os.path.join(CSRC, f), "-o", o])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    objs = [os.path.join(BUILD, f + ".o") for f in CXX_SOURCES + CU_SOURCES]
    tmp = OUT + ".tmp"
    logs.append(_run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]))
    os.replace(tmp, OUT)
    if verbose:
        print("".join(logs))
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
