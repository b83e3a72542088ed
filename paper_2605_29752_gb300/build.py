"""Build the C-ABI library librg.so in-tree for sm_103a.

CUDA sources are compiled by nvcc for `-gencode arch=compute_103a,code=sm_103a`,
host C++ by g++ (no floating-point contraction, no fast-math: the statistics
and the plan tables are bit-exact by construction), all translation units in
parallel.  The CUDA runtime is linked statically and the driver API is reached
through cudaGetDriverEntryPointByVersion, so the library loads (and exports its
symbols) on a machine without a GPU or driver.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librg.so")
LIB_TIMERS = os.path.join(PKG, "librg_timers.so")

CUDA_SOURCES = ["rg_gemm.cu", "rg_fp8.cu", "rg_grouped.cu"]
CXX_SOURCES = ["rg_plan.cpp", "rg_stats.cpp", "rg_serve.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_include(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def commands(debug: bool = False, phase_timers: bool = False):
    nvcc = _nvcc()
    cinc = _cuda_include(nvcc)
    opt = ["-O0", "-g"] if debug else ["-O3"]
    build_dir = BUILD + ("_timers" if phase_timers else "")
    lib = LIB_TIMERS if phase_timers else LIB
    defs = ["-DRG_PHASE_TIMERS=1"] if phase_timers else []
    cmds = []
    objs = []
    for src in CUDA_SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(build_dir, src + ".o")
        cmds.append([nvcc, *ARCH, *opt, *defs, "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC, "-c", path, "-o", obj])
        objs.append(obj)
    for src in CXX_SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(build_dir, src + ".o")
        cmds.append(["g++", *opt, "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-Wall",
                     "-I", INCLUDE, "-I", CSRC, "-I", cinc, "-pthread", "-c", path, "-o", obj])
        objs.append(obj)
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", lib, *objs, "-lpthread", "-ldl", "-lrt"]
    return cmds, link, build_dir, lib


def build(verbose: bool = False, debug: bool = False, phase_timers: bool = False) -> str:
    """Build librg.so (or, with phase_timers, the instrumented librg_timers.so beside it)."""
    cmds, link, build_dir, lib = commands(debug, phase_timers)
    os.makedirs(build_dir, exist_ok=True)
    procs = []
    for c in cmds:
        if verbose:
            print(" ".join(c), flush=True)
        procs.append((c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for c, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((c, out))
        elif verbose and out.strip():
            print(out, flush=True)
    if failed:
        msg = "\n\n".join(" ".join(c) + "\n" + out for c, out in failed)
        raise RuntimeError("librg build failed:\n" + msg)
    tmp = lib + ".tmp"
    link = [tmp if x == lib else x for x in link]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("librg link failed:\n" + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv, phase_timers="--phase-timers" in sys.argv))
