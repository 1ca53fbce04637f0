"""Build the CUDA library libhlbm.so (sm_103a) in-tree.

    python -m paper_2510_13726_b300.build [--force] [--verbose]

Compiles the kernels and the C ABI (include/hlbm.h) with nvcc for
``-gencode arch=compute_103a,code=sm_103a``.  Host code keeps IEEE semantics
(no FMA contraction) because the rotor frames are rounded on the host.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(CSRC, f) for f in ("hl_kernels.cu", "hl_api.cu", "hl_grad.cu", "hl_noalloc.cu")]
HEADERS = [os.path.join(CSRC, f) for f in ("hl_device.cuh", "hl_adjoint.cuh", "hl_pair.cuh", "hl_internal.h", "hl_host.h")] + [
    os.path.join(ROOT, "include", "hlbm.h")]
LIB = os.path.join(HERE, "libhlbm.so")
NVCC = os.environ.get("NVCC", "nvcc")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile each source to an object file (in parallel), then link."""
    if not force and not _stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
             "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags += ["-Xptxas", "-v"]
    objs = [os.path.join(objdir, os.path.splitext(os.path.basename(src))[0] + ".o") for src in SOURCES]

    def compile_one(k):
        subprocess.run(flags + ["-c", SOURCES[k], "-o", objs[k]], check=True)

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(compile_one, range(len(SOURCES))))
    tmp = LIB + ".tmp"
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
