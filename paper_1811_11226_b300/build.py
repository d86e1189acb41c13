"""Build libaugwarp.so (the CUDA library behind include/augwarp.h) in-tree.

Compiles every ``csrc/*.cu`` for sm_103a only (``-gencode
arch=compute_103a,code=sm_103a``), in parallel, and links them with the CUDA
runtime into ``paper_1811_11226_b300/libaugwarp.so``.  Rebuilds only when a
source or header is newer than the library.  No fast-math flags: the kernels
rely on exact IEEE float rounding of their arithmetic, and call the hardware
approximations (``lg2/sqrt/sin/cos.approx.ftz`` in the Box-Muller transform,
``ex2/lg2.approx`` in the loss variants) only through explicit inline PTX,
whose error bounds the kernels' comments state.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libaugwarp.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
         "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _obj(src: str) -> str:
    return os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")


def _obj_fresh(src: str) -> bool:
    """An object is reused when it is newer than its source and every header
    (headers are shared by all sources, so a header change rebuilds all)."""
    obj = _obj(src)
    if not os.path.exists(obj):
        return False
    t = os.path.getmtime(obj)
    headers = [p for p in _deps() if not p.endswith(".cu")]
    return all(os.path.getmtime(p) <= t for p in [src, *headers])


def _compile(src: str, verbose_ptxas: bool) -> str:
    obj = _obj(src)
    cmd = [NVCC, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    stale = [s for s in srcs if force or verbose_ptxas or not _obj_fresh(s)]
    if stale:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(stale))) as ex:
            list(ex.map(lambda s: _compile(s, verbose_ptxas), stale))
    objs = [_obj(s) for s in srcs]
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
