"""Plain CPU oracle for degree-binned wedge sampling (Kolda et al., "Counting
Triangles in Massive Graphs with MapReduce").

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(``paper_1301_5887_gb300``) never imports it and shares no code with it; the
one shared module is the seeded input generator ``graphgen``.

The arithmetic lives in ``oracle.c`` (each function cites the passage it
follows); this module marshals numpy arrays through ctypes. ``estimate`` and
``brute`` hold the FP64 estimators and the tiny-graph brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "..", "graphgen", "graphgen.h")]

STAT_BINS = 34  # BinId with tau=2, omega=2 of any degree < 2^31 is at most 32


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, OpenMP). Returns its path."""
    fresh = os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in _SRC)
    if fresh and not force:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp,
           os.path.join(_HERE, "oracle.c"), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u32, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        _lib.oracle_csr.argtypes = [i64, P, P, i32, P, P, P]
        _lib.oracle_csr.restype = ctypes.c_int
        _lib.oracle_bin_lodeg.argtypes = [u64, u32, u64]
        _lib.oracle_bin_lodeg.restype = u64
        _lib.oracle_bin_id.argtypes = [u64, u32, u64]
        _lib.oracle_bin_id.restype = u32
        _lib.oracle_bins.argtypes = [i32, P, u32, u64, i32, P, P]
        _lib.oracle_bins.restype = i32
        _lib.oracle_philox4x32_10.argtypes = [P, P, P]
        _lib.oracle_philox4x32_10.restype = None
        _lib.oracle_hoeffding_k.argtypes = [dbl, dbl]
        _lib.oracle_hoeffding_k.restype = u64
        _lib.oracle_sample.argtypes = [i32, P, P, u32, u64, i32, u64, u64, u64, P, P, P, P, P, u64]
        _lib.oracle_sample.restype = ctypes.c_int
        _lib.oracle_sample_rounding.argtypes = [i32, P, P, u32, u64, i32, u64, u64, P, P, P]
        _lib.oracle_sample_rounding.restype = ctypes.c_int
        _lib.oracle_classify.argtypes = [i32, P, P, u32, u64, i64, P, P, P, P]
        _lib.oracle_classify.restype = ctypes.c_int
        _lib.oracle_exact.argtypes = [i32, P, P, u32, u64, i32, P, P]
        _lib.oracle_exact.restype = u64
        _lib.oracle_rows_kronecker.argtypes = [u32, i64, dbl, dbl, dbl, u64, ctypes.c_int, i64, P, i64, P, P]
        _lib.oracle_rows_kronecker.restype = i64
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# --------------------------------------------------------------------------
# Graph
# --------------------------------------------------------------------------

def csr(src, dst, n: int):
    """Undirected simple graph of an edge list (union of directions, duplicates
    collapsed, self-loops dropped; Sec. 5.1). Returns (off[n+1] int64,
    adj[2m] int32) with each row ascending."""
    src = _c(src, np.int32)
    dst = _c(dst, np.int32)
    ne = src.shape[0]
    off = np.zeros(n + 1, np.int64)
    adj = np.zeros(max(2 * ne, 1), np.int32)
    m2 = ctypes.c_int64(0)
    rc = _L().oracle_csr(ne, _p(src), _p(dst), n, _p(off), _p(adj), ctypes.byref(m2))
    if rc == -1:
        raise ValueError("vertex id outside [0, n)")
    if rc != 0:
        raise MemoryError("oracle_csr failed")
    return off, adj[: m2.value].copy()


def degrees(off: np.ndarray) -> np.ndarray:
    return np.diff(off).astype(np.int64)


# --------------------------------------------------------------------------
# Binning (Sec. 4.2)
# --------------------------------------------------------------------------

def bin_lodeg(k: int, tau: int, omega: int) -> int:
    return int(_L().oracle_bin_lodeg(k, tau, omega))


def bin_id(d: int, tau: int, omega: int) -> int:
    return int(_L().oracle_bin_id(d, tau, omega))


def n_bins_for(off: np.ndarray, tau: int, omega: int) -> int:
    """Array length that indexes every bin id present (bin ids start at 1)."""
    dmax = int(degrees(off).max()) if off.shape[0] > 1 else 0
    return max(bin_id(max(dmax, 1), tau, omega) + 1, 2)


def bins(off: np.ndarray, tau: int, omega: int):
    """Alg. Phase 1b: n_b and p_b indexed by bin id."""
    off = _c(off, np.int64)
    n = off.shape[0] - 1
    nb = n_bins_for(off, tau, omega)
    n_b = np.zeros(nb, np.uint64)
    p_b = np.zeros(nb, np.uint64)
    rc = _L().oracle_bins(n, _p(off), tau, omega, nb, _p(n_b), _p(p_b))
    if rc < 0:
        raise RuntimeError("oracle_bins: bin table too small")
    lo = np.array([bin_lodeg(k, tau, omega) for k in range(nb + 1)], dtype=np.uint64)
    return {"n_bins": nb, "n_b": n_b, "p_b": p_b, "lo": lo[:nb], "hi": lo[1:] - np.uint64(1)}


# --------------------------------------------------------------------------
# Random words, budget
# --------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _L().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def hoeffding_k(eps: float, delta: float) -> int:
    """Thm 3.1: smallest k >= 0.5 eps^-2 ln(2/delta)."""
    return int(_L().oracle_hoeffding_k(eps, delta))


# --------------------------------------------------------------------------
# Sampling, classification, exact counts
# --------------------------------------------------------------------------

def sample(off, adj, tau: int, omega: int, seed: int, k_per_bin: int, k_global: int, records: bool = False,
           k_bins=None, first: int = 0):
    """Per-bin and global wedge sampling (Thm 3.2, Thm 3.3, Sec. 3.2) with the
    tally of Alg. Phase 4c. Returns counts[n_bins, 5] = (k_b, q0, q1, q2, q3),
    glob = (k_global, closed), stats[34, 34] and optional records[k_global, 8].
    k_bins (optional, indexed by bin id) gives each bin its own budget; every
    stream draws sample indices first .. first + k - 1."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    n = off.shape[0] - 1
    nb = n_bins_for(off, tau, omega)
    counts = np.zeros((nb, 5), np.uint64)
    glob = np.zeros(2, np.uint64)
    stats = np.zeros((STAT_BINS, STAT_BINS), np.uint64)
    rec = np.zeros((k_global, 8), np.int32) if records else None
    kb = None
    if k_bins is not None:
        kb = np.zeros(nb, np.uint64)
        src = np.asarray(k_bins, dtype=np.uint64)
        kb[: min(nb, src.shape[0])] = src[:nb]
    rc = _L().oracle_sample(n, _p(off), _p(adj), tau, omega, nb, seed, k_per_bin, k_global, _p(counts), _p(glob),
                            _p(stats), _p(rec) if records else ctypes.c_void_p(0),
                            _p(kb) if kb is not None else ctypes.c_void_p(0), first)
    if rc != 0:
        raise RuntimeError(f"oracle_sample failed ({rc})")
    return {"counts": counts, "glob": glob, "stats": stats, "records": rec}


def sample_rounding(off, adj, tau: int, omega: int, seed: int, k_per_bin: int, k_bins=None, per_vertex=False):
    """Per-bin samples allocated per vertex by probabilistic rounding (Alg.
    Phase 2a) and drawn per centre (Alg. Phase 2c). Returns counts[n_bins, 5]
    = (realised k_b, q0, q1, q2, q3) and, with per_vertex, q_v for every vertex."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    n = off.shape[0] - 1
    nb = n_bins_for(off, tau, omega)
    counts = np.zeros((nb, 5), np.uint64)
    qv = np.zeros(n, np.uint64) if per_vertex else None
    kb = None
    if k_bins is not None:
        kb = np.zeros(nb, np.uint64)
        src = np.asarray(k_bins, dtype=np.uint64)
        kb[: min(nb, src.shape[0])] = src[:nb]
    rc = _L().oracle_sample_rounding(n, _p(off), _p(adj), tau, omega, nb, seed, k_per_bin,
                                     _p(kb) if kb is not None else ctypes.c_void_p(0), _p(counts),
                                     _p(qv) if per_vertex else ctypes.c_void_p(0))
    if rc != 0:
        raise RuntimeError(f"oracle_sample_rounding failed ({rc})")
    return {"counts": counts, "qv": qv}


def classify(off, adj, tau: int, omega: int, v0, v1, v2):
    """Closure + q-class of the given wedges (Alg. Phase 3b, Alg. Phase 4c)."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    v0, v1, v2 = _c(v0, np.int32), _c(v1, np.int32), _c(v2, np.int32)
    q = np.zeros(v0.shape[0], np.uint8)
    rc = _L().oracle_classify(off.shape[0] - 1, _p(off), _p(adj), tau, omega, v0.shape[0], _p(v0), _p(v1), _p(v2),
                              _p(q))
    if rc != 0:
        raise ValueError("wedge vertex outside [0, n)")
    return q


def exact(off, adj, tau: int, omega: int):
    """Exact t, t_i and p_{b,q} by triangle enumeration (Sec. 2.1, 2.2).
    pbq[b, 0] = p_b - sum_{q>=1} p_{b,q}."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    n = off.shape[0] - 1
    nb = n_bins_for(off, tau, omega)
    t_i = np.zeros(max(n, 1), np.uint64)
    pbq = np.zeros((nb, 4), np.uint64)
    t = int(_L().oracle_exact(n, _p(off), _p(adj), tau, omega, nb, _p(t_i), _p(pbq)))
    if t == 2**64 - 1:
        raise MemoryError("oracle_exact failed")
    bb = bins(off, tau, omega)
    pbq[:, 0] = bb["p_b"] - pbq[:, 1:].sum(axis=1)
    return {"t": t, "t_i": t_i[:n], "pbq": pbq, "n_b": bb["n_b"], "p_b": bb["p_b"]}


def rows_kronecker(scale: int, n_edges: int, a: float, b: float, c: float, seed: int, permute: bool, query,
                   cap: int = 1 << 24):
    """Exact neighbour sets of the query vertices of a generated Kronecker graph,
    by one scan over its generated edges. Returns {vertex: ascending int32 array}."""
    q = np.unique(_c(query, np.int32))
    nq = q.shape[0]
    while True:
        pq = np.zeros(cap, np.int32)
        pn = np.zeros(cap, np.int32)
        total = int(_L().oracle_rows_kronecker(scale, n_edges, a, b, c, seed, int(permute), nq, _p(q), cap, _p(pq),
                                               _p(pn)))
        if total <= cap:
            break
        cap = total
    key = pq[:total].astype(np.int64) << 32 | pn[:total].astype(np.int64)
    key = np.unique(key)
    qi = (key >> 32).astype(np.int64)
    nb = (key & 0xFFFFFFFF).astype(np.int32)
    bounds = np.searchsorted(qi, np.arange(nq + 1))
    return {int(v): nb[bounds[i]:bounds[i + 1]].copy() for i, v in enumerate(q)}
