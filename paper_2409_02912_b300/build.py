"""Build the CUDA library ``libnrx.so`` in-tree for sm_103a (B300).

Usage: ``python -m paper_2409_02912_b300.build`` (or ``build()`` from Python).
Cross-compiles with nvcc; no GPU is needed to build.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libnrx.so")
BUILD_DIR = os.path.join(PKG, "_build")
# bounds-checked variant: every instrumented kernel index checked, violations
# counted (nrx_debug_counters) and their accesses skipped
LIB_DEBUG = os.path.join(PKG, "libnrx_debug.so")
BUILD_DIR_DEBUG = os.path.join(PKG, "_build_debug")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(PKG, "..", "include", "*.h"))
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile every ``csrc/*.cu`` and link ``libnrx.so`` (with ``debug``, the
    bounds-checked ``libnrx_debug.so``, built with -DNRX_DEBUG); returns its
    path."""
    bdir, lib = (BUILD_DIR_DEBUG, LIB_DEBUG) if debug else (BUILD_DIR, LIB)
    os.makedirs(bdir, exist_ok=True)
    objs = []
    changed = False
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if _stale(obj, src) or ptxas_info:
            cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *(["-DNRX_DEBUG"] if debug else []), "-c", src, "-o", obj]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0 or verbose or ptxas_info:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}")
            changed = True
    if changed or not os.path.exists(lib):
        cmd = [nvcc(), *ARCH, "-shared", "-o", lib, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_info="--ptxas-info" in sys.argv, debug="--debug" in sys.argv))
