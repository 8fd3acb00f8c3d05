"""Build libmerf.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libmerf.so")
LIB_DEBUG = os.path.join(PKG, "libmerf_debug.so")   # bounds-checked build (-DMERF_DEBUG_BOUNDS)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
              "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile the library (debug: the bounds-checked build) and return its path."""
    out = LIB_DEBUG if debug else LIB
    if not force and not ptxas_info and up_to_date(out):
        return out
    nvcc = os.environ.get("NVCC", "nvcc")
    extra = ["-DMERF_DEBUG_BOUNDS"] if debug else []
    tag = f"{os.getpid()}"
    objs, procs = [], []
    # each translation unit compiles in its own nvcc process, in parallel; one link step follows
    for src in sources():
        obj = os.path.join(PKG, os.path.basename(src) + f".{tag}{'.dbg' if debug else ''}.o")
        cmd = [nvcc, *ARCH, *[f for f in NVCC_FLAGS if f != "-shared"], *extra, "-I", INCLUDE, "-I", CSRC, "-c",
               "-o", obj, src]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        objs.append(obj)
        procs.append(subprocess.Popen(cmd))
    try:
        failed = [p.wait() for p in procs]
        if any(failed):
            raise subprocess.CalledProcessError(max(failed), "nvcc")
        tmp = out + f".{tag}.tmp"
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, out)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return out


if __name__ == "__main__":
    build(force=True, verbose=True, ptxas_info="-v" in sys.argv, debug="--debug" in sys.argv)
