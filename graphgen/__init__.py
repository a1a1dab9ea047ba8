"""Seeded synthetic graph generators (input generation only).

The one module shared by the CPU oracle and the device path: both consume the
edge lists it produces. It holds none of the wedge-sampling arithmetic.
``kronecker_host``/``chunglu_host`` write host arrays (gen_host.c);
``kronecker_device``/``chunglu_device`` write device buffers (gen_cuda.cu) and
produce exactly the same edges.

Workload of the paper's synthetic graphs (Sec. 5.1): Graph500 Kronecker with
generator matrix [0.57 0.19; 0.19 0.05], edge factor 16, permuted vertex ids.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libgraphgen_host.so")
_CUDA_SO = os.path.join(_HERE, "libgraphgen_cuda.so")
_HDR = os.path.join(_HERE, "graphgen.h")

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19
EDGEFACTOR = 16


def _fresh(so, srcs):
    return os.path.exists(so) and all(os.path.getmtime(so) >= os.path.getmtime(s) for s in srcs)


def build_host(force: bool = False) -> str:
    src = os.path.join(_HERE, "gen_host.c")
    if force or not _fresh(_HOST_SO, [src, _HDR]):
        tmp = _HOST_SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o",
                        tmp, src, "-lm"],
                       check=True)
        os.replace(tmp, _HOST_SO)
    return _HOST_SO


def build_cuda(force: bool = False) -> str:
    src = os.path.join(_HERE, "gen_cuda.cu")
    if force or not _fresh(_CUDA_SO, [src, _HDR]):
        tmp = _CUDA_SO + f".tmp{os.getpid()}"
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-shared", "-o", tmp, src], check=True)
        os.replace(tmp, _CUDA_SO)
    return _CUDA_SO


def build(force: bool = False):
    return build_host(force), build_cuda(force)


_host = None
_cuda = None


def _H():
    global _host
    if _host is None:
        _host = ctypes.CDLL(build_host())
        P, i64, u32, u64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        _host.graphgen_kronecker_host.argtypes = [u32, i64, i64, dbl, dbl, dbl, u64, ctypes.c_int, P, P]
        _host.graphgen_kronecker_host.restype = ctypes.c_int
        _host.graphgen_chunglu_weights.argtypes = [u64, dbl, dbl, P]
        _host.graphgen_chunglu_weights.restype = i64
        _host.graphgen_chunglu_host.argtypes = [P, u64, i64, i64, u64, ctypes.c_int, P, P]
        _host.graphgen_chunglu_host.restype = ctypes.c_int
        _host.graphgen_rmat_noisy_levels.argtypes = [u32, dbl, dbl, dbl, dbl, u64, P]
        _host.graphgen_rmat_noisy_levels.restype = ctypes.c_int
        _host.graphgen_kronecker_levels_host.argtypes = [u32, i64, i64, P, u64, ctypes.c_int, P, P]
        _host.graphgen_kronecker_levels_host.restype = ctypes.c_int
        _host.graphgen_permute_host.argtypes = [u64, u64, i64, P, P]
        _host.graphgen_permute_host.restype = ctypes.c_int
    return _host


def _D():
    global _cuda
    if _cuda is None:
        _cuda = ctypes.CDLL(build_cuda())
        P, i64, u32, u64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        _cuda.graphgen_kronecker_device.argtypes = [u32, i64, dbl, dbl, dbl, u64, ctypes.c_int, P, P, P]
        _cuda.graphgen_kronecker_device.restype = ctypes.c_int
        _cuda.graphgen_kronecker_levels_device.argtypes = [u32, i64, P, u64, ctypes.c_int, P, P, P]
        _cuda.graphgen_kronecker_levels_device.restype = ctypes.c_int
        _cuda.graphgen_chunglu_device.argtypes = [P, u64, i64, u64, ctypes.c_int, P, P, P]
        _cuda.graphgen_chunglu_device.restype = ctypes.c_int
    return _cuda


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def kronecker_edges(scale: int, edgefactor: int = EDGEFACTOR) -> int:
    return edgefactor << scale


def rmat_levels(scale: int, noise: float, seed: int = 1, a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C):
    """Integer quadrant thresholds (scale, 3) of the noisy SKG levels (noise 0: the plain matrix at every level)."""
    th = np.zeros((scale, 3), np.uint32)
    if _H().graphgen_rmat_noisy_levels(scale, a, b, c, noise, seed, _ptr(th)) != 0:
        raise ValueError("graphgen_rmat_noisy_levels: bad arguments")
    return th


def kronecker_host(scale: int, n_edges: int | None = None, seed: int = 1, permute: bool = True,
                   a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C, e0: int = 0, noise: float = 0.0):
    """Edges [e0, e0 + n_edges) of the R-MAT graph with 2^scale vertices (host int32 arrays).
    noise > 0: noisy SKG with that noise parameter (the paper uses 0.1)."""
    if n_edges is None:
        n_edges = kronecker_edges(scale)
    src = np.empty(n_edges, np.int32)
    dst = np.empty(n_edges, np.int32)
    if noise > 0:
        th = rmat_levels(scale, noise, seed, a, b, c)
        rc = _H().graphgen_kronecker_levels_host(scale, e0, e0 + n_edges, _ptr(th), seed, int(permute), _ptr(src),
                                                 _ptr(dst))
    else:
        rc = _H().graphgen_kronecker_host(scale, e0, e0 + n_edges, a, b, c, seed, int(permute), _ptr(src),
                                          _ptr(dst))
    if rc != 0:
        raise ValueError("graphgen_kronecker_host: bad arguments")
    return src, dst


def kronecker_device(scale: int, src_ptr: int, dst_ptr: int, n_edges: int, stream_ptr: int = 0, seed: int = 1,
                     permute: bool = True, a: float = RMAT_A, b: float = RMAT_B, c: float = RMAT_C,
                     noise: float = 0.0):
    """Same edges as kronecker_host, written to device buffers (raw pointers)."""
    if noise > 0:
        th = rmat_levels(scale, noise, seed, a, b, c)
        rc = _D().graphgen_kronecker_levels_device(scale, n_edges, _ptr(th), seed, int(permute),
                                                   ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr),
                                                   ctypes.c_void_p(stream_ptr))
    else:
        rc = _D().graphgen_kronecker_device(scale, n_edges, a, b, c, seed, int(permute), ctypes.c_void_p(src_ptr),
                                            ctypes.c_void_p(dst_ptr), ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError(f"graphgen_kronecker_device failed (cudaError {rc})")


def chunglu_weights(n: int, gamma: float, mean_deg: float):
    """Integer weight prefix (uint64[n]) and edge count of a Chung-Lu graph."""
    prefix = np.empty(n, np.uint64)
    m = _H().graphgen_chunglu_weights(n, gamma, mean_deg, _ptr(prefix))
    if m < 0:
        raise ValueError("graphgen_chunglu_weights: bad arguments")
    return prefix, int(m)


def chunglu_host(prefix, n_edges: int, seed: int, permute: bool = True, e0: int = 0):
    prefix = np.ascontiguousarray(prefix, dtype=np.uint64)
    src = np.empty(n_edges, np.int32)
    dst = np.empty(n_edges, np.int32)
    rc = _H().graphgen_chunglu_host(_ptr(prefix), prefix.shape[0], e0, e0 + n_edges, seed, int(permute), _ptr(src),
                                    _ptr(dst))
    if rc != 0:
        raise ValueError("graphgen_chunglu_host: bad arguments")
    return src, dst


def chunglu_device(prefix_dev_ptr: int, n: int, src_ptr: int, dst_ptr: int, n_edges: int, seed: int,
                   permute: bool = True, stream_ptr: int = 0):
    rc = _D().graphgen_chunglu_device(ctypes.c_void_p(prefix_dev_ptr), n, n_edges, seed, int(permute),
                                      ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr), ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError(f"graphgen_chunglu_device failed (cudaError {rc})")


def permute_host(n: int, seed: int, x):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    y = np.empty_like(x)
    rc = _H().graphgen_permute_host(n, seed, x.shape[0], _ptr(x), _ptr(y))
    if rc != 0:
        raise ValueError("graphgen_permute_host: bad arguments")
    return y
