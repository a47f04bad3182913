"""Build libffadmm.so in-tree (sm_103a only).

Each translation unit is compiled in parallel; host C++ (the setup-time
factorization) goes through g++, CUDA sources through nvcc with
-gencode arch=compute_103a,code=sm_103a.  The result lands next to this file.
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
LIB = os.path.join(HERE, "libffadmm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["ffa_api.cu", "ffa_local.cu", "ffa_solve.cu", "ffa_adjoint.cu", "ffa_noalloc.cu", "ffa_devfactor.cu",
              "ffa_topinv.cu"]
CXX_SOURCES = ["ffa_factor.cpp", "ffa_schedule.cpp", "ffa_state.cpp", "ffa_constraint_host.cpp",
               "ffa_operator_host.cpp", "ffa_devfactor_plan.cpp", "ffa_topinv_plan.cpp"]
# The per-element kernels' float divisions and square roots (Newton steps of the
# prox roots, Jacobi rotation parameters, normalizations) take the hardware's
# approximate forms: each is followed by iterations or renormalizations that
# absorb a few ulp, and the local step is issue bound (0.169 -> 0.154 ms on the
# 1.57M-tet cube).  Double precision is not affected by these options.
PER_FILE_FLAGS = {"ffa_local.cu": ["-prec-div=false", "-prec-sqrt=false"]}


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libffadmm")
    return cand


def _run(cmd: list[str]) -> None:
    proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + proc.stdout)


def _stale(obj: str, src: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "ffadmm.h"))
    headers.append(os.path.abspath(__file__))   # compile options live here
    jobs, objs = [], []
    for f in CU_SOURCES:
        src, obj = os.path.join(CSRC, f), os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _stale(obj, src, headers):
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                         *PER_FILE_FLAGS.get(f, []), "-c", src, "-o", obj])
    for f in CXX_SOURCES:
        src, obj = os.path.join(CSRC, f), os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _stale(obj, src, headers):
            jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
            for fut in [ex.submit(_run, j) for j in jobs]:
                fut.result()
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
