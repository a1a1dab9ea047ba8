"""Build libwedge.so (the C-ABI library) in-tree for sm_103a with nvcc.

Each csrc/*.cu is compiled in parallel to an object under _build/, then the
objects are linked into paper_1301_5887_gb300/libwedge.so with the CUDA
runtime linked statically. The same sources compiled with
-DWEDGE_DEBUG_BOUNDS give libwedge_debug.so (objects under _build_debug/):
index checks at the kernels' gathered-offset accesses that record an error
instead of faulting, the stand-in for a memory checker. Rebuilds only when a
source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
SO = os.path.join(PKG, "libwedge.so")
OUT_DEBUG = os.path.join(PKG, "_build_debug")
SO_DEBUG = os.path.join(PKG, "libwedge_debug.so")
HEADER = os.path.join(ROOT, "include", "wedge.h")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                  "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + [HEADER,
                                                                                                        __file__]


def fresh(so: str = SO) -> bool:
    if not os.path.exists(so):
        return False
    t = os.path.getmtime(so)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src: str, verbose: bool, outdir: str, extra) -> str:
    obj = os.path.join(outdir, os.path.basename(src)[:-3] + ".o")
    cmd = ["nvcc"] + NVFLAGS + list(extra) + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libwedge.so and libwedge_debug.so (all translation
    units of both in parallel); returns the path of libwedge.so."""
    todo = [(so, out, extra) for so, out, extra in ((SO, OUT, ()), (SO_DEBUG, OUT_DEBUG, ("-DWEDGE_DEBUG_BOUNDS",)))
            if force or not fresh(so)]
    if not todo:
        return SO
    srcs = sources()
    jobs = []
    for so, out, extra in todo:
        os.makedirs(out, exist_ok=True)
        jobs += [(src, out, extra) for src in srcs]
    with ThreadPoolExecutor(max_workers=min(len(jobs), max(os.cpu_count() or 4, 4))) as ex:
        objs = list(ex.map(lambda j: _compile(j[0], verbose, j[1], j[2]), jobs))
    for so, out, extra in todo:
        mine = [o for o in objs if os.path.dirname(o) == out]
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["nvcc"] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + mine
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, so)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
