"""Builds libwvl.so in-tree for sm_103a with nvcc (no cmake, parallel TUs).

Used by ``__graft_entry__.build()`` and by the package loader when the
library is missing or older than its sources.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwvl.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["api.cu", "kernels_f64.cu", "kernels_f32.cu", "emu_kernel.cu", "fused_kernel.cu",
              "reduce.cu", "noalloc.cu", "pcg.cu", "probe.cu", "overlap.cu"]
CPP_SOURCES = ["filters.cpp"]
HEADERS = ["wvl_internal.h", "taps.h", "pass_kernel.cuh", "kernels_impl.cuh", "emu.cuh"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwvl.so")


def _sources():
    return ([os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES + HEADERS]
            + [os.path.join(INCLUDE, "wvl.h"), os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    common = ["-std=c++17", "-O3", "-I", INCLUDE, "-I", CSRC]
    cmds = []
    objs = []
    for s in CU_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        objs.append(o)
        cmd = [nv, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-c", os.path.join(CSRC, s), "-o", o]
        if verbose or os.environ.get("WVL_PTXAS_VERBOSE"):
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
    for s in CPP_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        objs.append(o)
        cmds.append([nv, *common, "-x", "c++", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-c", os.path.join(CSRC, s), "-o", o])
    with ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        outs = list(ex.map(_run, cmds))
    tmp = LIB + ".tmp"
    _run([nv, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
