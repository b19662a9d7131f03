"""Compile the CUDA library libprop.so in-tree for sm_103a (nvcc, no cmake).

``python -m paper_2410_17446_gb300.build`` or ``build()``; rebuilds only when a
source is newer than the library.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = [os.path.join(PKG, "csrc", f) for f in ("prop.cu", "prop_mg.cu", "cnn.cu")]
DEPS = SRC + [os.path.join(PKG, "csrc", f) for f in ("fft.cuh", "kernels.cuh", "mg.cuh", "tma.cuh")] + [
    os.path.join(ROOT, "include", h) for h in ("prop.h", "prop_cnn.h")]
LIB = os.path.join(PKG, "libprop.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile each translation unit in parallel, then link libprop.so."""
    if not force and not needs_build():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    objs = [os.path.join(PKG, "_obj_" + os.path.basename(s) + ".o") for s in SRC]
    # PROP_NVCC_FLAGS: extra nvcc flags (e.g. -DPROP_SYNC_EVERY=8 to try another batch length)
    flags = ["-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             *os.environ.get("PROP_NVCC_FLAGS", "").split()]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc(), *flags, "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), flush=True)
        return subprocess.run(cmd, capture_output=True, text=True)

    with ThreadPoolExecutor(len(SRC)) as ex:
        results = list(ex.map(compile_one, zip(SRC, objs)))
    for r in results:
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed ({r.returncode}):\n{r.stdout}\n{r.stderr}")
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed ({r.returncode}):\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
