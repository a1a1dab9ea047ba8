"""Python binding of libwedge.so, the GB300 wedge-sampling library.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels behind the C ABI declared in include/wedge.h. The functions keep
the C names without the ``wedge_`` prefix:

    graph_build(src, dst, n_vertices, stream) -> Graph      (wedge_graph_build)
    bin(graph, tau, omega, stream) -> Bins                  (wedge_bin)
    sample(graph, bins, seed, eps, delta, k_per_bin, k_global, ...) -> Counts
    estimate(counts, delta) -> dict                         (wedge_estimate)
    classify(graph, bins, v0, v1, v2, q, stream)            (wedge_classify)
    hoeffding_k(eps, delta)

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; host arrays are
copied to the device inside the library. PyTorch supplies device memory and
streams only. If libwedge.so is missing the import of the library fails
loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_PKG, "libwedge.so")

MAX_BINS = 256
STAT_BINS = 34
FLAG_NO_GLOBAL = 0x1
FLAG_NO_BINS = 0x2
FLAG_ROUNDING = 0x4  # per-bin samples allocated per vertex by probabilistic rounding (Alg. Phase 2a)
FLAG_SORTED_CLOSURE = 0x8  # per-bin closure queries radix-sorted, then checked in order (Alg. Phase 3b join)

STATUS = {0: "WEDGE_OK", 1: "WEDGE_EINVAL", 2: "WEDGE_ENOMEM", 3: "WEDGE_ECUDA", 4: "WEDGE_ETIMEOUT",
          5: "WEDGE_EOVERFLOW", 6: "WEDGE_EBUSY"}
EBUSY = 6


class WedgeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


# ---------------------------------------------------------------------------
# ABI structs (mirror include/wedge.h)
# ---------------------------------------------------------------------------
_vp = ctypes.c_void_p


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("id_bits", ctypes.c_int32), ("n_adj", ctypes.c_int64),
                ("n_input_edges", ctypes.c_int64), ("max_degree", ctypes.c_int32), ("off", _vp), ("adj", _vp),
                ("deg", _vp)]


class BinParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_uint32), ("omega", ctypes.c_uint64)]


class BinsInfo(ctypes.Structure):
    _fields_ = [("n_bins", ctypes.c_uint32), ("tau", ctypes.c_uint32), ("omega", ctypes.c_uint64),
                ("lo_deg", ctypes.c_uint64 * MAX_BINS), ("hi_deg", ctypes.c_uint64 * MAX_BINS),
                ("n_b", ctypes.c_uint64 * MAX_BINS), ("p_b", ctypes.c_uint64 * MAX_BINS),
                ("start", ctypes.c_int64 * (MAX_BINS + 1)), ("p_total", ctypes.c_uint64),
                ("n_wedge_vertices", ctypes.c_int64), ("L", _vp), ("W", _vp)]


class SampleParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("eps", ctypes.c_double), ("delta", ctypes.c_double),
                ("k_per_bin", ctypes.c_uint64), ("k_global", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("records", _vp), ("k_bin", _vp), ("first_sample", ctypes.c_uint64)]


class Record(ctypes.Structure):
    _fields_ = [(x, ctypes.c_int32) for x in ("v0", "v1", "v2", "closed", "d0", "d1", "d2", "reserved")]


class CountsStruct(ctypes.Structure):
    _fields_ = [("n_bins", ctypes.c_uint32), ("k_b", ctypes.c_uint64 * MAX_BINS),
                ("q", (ctypes.c_uint64 * 4) * MAX_BINS), ("n_b", ctypes.c_uint64 * MAX_BINS),
                ("p_b", ctypes.c_uint64 * MAX_BINS), ("p_total", ctypes.c_uint64), ("k_global", ctypes.c_uint64),
                ("closed_global", ctypes.c_uint64), ("stats", (ctypes.c_uint64 * STAT_BINS) * STAT_BINS)]


class EstimatesStruct(ctypes.Structure):
    _fields_ = [("n_bins", ctypes.c_uint32), ("c_b", ctypes.c_double * MAX_BINS), ("t_b", ctypes.c_double * MAX_BINS),
                ("eps_b", ctypes.c_double * MAX_BINS), ("p_total", ctypes.c_double), ("c_hat", ctypes.c_double),
                ("t_hat", ctypes.c_double), ("c_hat_global", ctypes.c_double), ("t_hat_global", ctypes.c_double),
                ("eps_global", ctypes.c_double)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("first_start_ms", ctypes.c_double), ("last_end_ms", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("graph", _vp), ("bins", _vp), ("params", SampleParams)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("mapping_small", ctypes.c_uint32), ("mapping_medium", ctypes.c_uint32),
                ("mapping_large", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("samples_per_tile", ctypes.c_uint32), ("flags", ctypes.c_uint32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


MAP_THREAD = 1
MAP_WARP = 2
BATCH_DIRECT = 1


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("max_batch_requests", ctypes.c_uint32), ("tau", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("omega", ctypes.c_uint64), ("launch", LaunchConfig), ("max_batch_samples", ctypes.c_uint64),
                ("max_queued_samples", ctypes.c_uint64), ("gpu_filling_samples", ctypes.c_uint64)]


class ServerRequest(ctypes.Structure):
    _fields_ = [("graph_id", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("eps", ctypes.c_double),
                ("delta", ctypes.c_double), ("k_per_bin", ctypes.c_uint64), ("k_global", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class RequestTiming(ctypes.Structure):
    _fields_ = [("submit_us", ctypes.c_double), ("dispatch_us", ctypes.c_double), ("done_us", ctypes.c_double),
                ("batch_requests", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ServerMetrics(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("samples", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("mean_batch_requests", ctypes.c_double), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double), ("span_s", ctypes.c_double),
                ("resident_graphs", ctypes.c_uint32), ("queued", ctypes.c_uint32),
                ("inflight_batches", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("resident_bytes", ctypes.c_uint64), ("evictions", ctypes.c_uint64),
                ("rejected_uploads", ctypes.c_uint64), ("rejected_requests", ctypes.c_uint64),
                ("queued_samples", ctypes.c_uint64)]


class TriangleBox(ctypes.Structure):
    _fields_ = [(x, ctypes.c_uint64) for x in ("count", "min", "q1", "median", "q3", "max", "whisker_lo",
                                                "whisker_hi", "outliers")]


class TriangleSummary(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint64), ("closed", ctypes.c_uint64), ("box", TriangleBox * STAT_BINS),
                ("ratio_q", ctypes.c_double * 5), ("hist", (ctypes.c_uint64 * STAT_BINS) * STAT_BINS)]


class ExactCounts(ctypes.Structure):
    _fields_ = [("triangles", ctypes.c_uint64), ("n_bins", ctypes.c_uint32), ("p_total", ctypes.c_uint64),
                ("p_b", ctypes.c_uint64 * MAX_BINS), ("pbq", (ctypes.c_uint64 * 4) * MAX_BINS)]


_STRUCTS = [GraphInfo, BinsInfo, SampleParams, Record, CountsStruct, EstimatesStruct, KernelStat, Request,
            LaunchConfig, ServerConfig, ServerRequest, RequestTiming, ServerMetrics, TriangleBox, TriangleSummary,
            ExactCounts]

# Every symbol include/wedge.h declares.
EXPORTS = ["wedge_status_str", "wedge_last_error", "wedge_version", "wedge_abi_sizes", "wedge_graph_build",
           "wedge_graph_free", "wedge_graph_get_info", "wedge_graph_copy", "wedge_bin", "wedge_bins_free",
           "wedge_bins_get_info", "wedge_bins_copy", "wedge_sample", "wedge_hoeffding_k", "wedge_estimate", "wedge_classify",
           "wedge_profile_enable", "wedge_profile_reset", "wedge_profile_read", "wedge_trim",
           "wedge_degree_offsets_noalloc", "wedge_batch_create", "wedge_batch_launch", "wedge_batch_results",
           "wedge_batch_free", "wedge_batch_info", "wedge_sample_batch", "wedge_autotune", "wedge_server_create",
           "wedge_server_destroy", "wedge_server_add_graph", "wedge_server_remove_graph", "wedge_server_submit",
           "wedge_server_wait", "wedge_server_stats", "wedge_probe_random_read", "wedge_triangle_stats",
           "wedge_exact", "wedge_pool_used_bytes", "wedge_test_fail_allocation", "wedge_test_lookback_timeout",
           "wedge_graph_from_csr"]

_lib = None


def library_path() -> str:
    return _SO


def load():
    """Load libwedge.so (built by build.py / __graft_entry__.build()). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise ImportError(f"libwedge.so is not built ({_SO}); run __graft_entry__.build() — there is no CPU fallback")
    _lib = _configure(ctypes.CDLL(_SO))
    return _lib


_lib_debug = None


def load_debug():
    """The bounds-checked build, libwedge_debug.so (same C ABI; index checks
    at gathered-offset accesses report WEDGE_ECUDA instead of faulting). Its
    handles must not be mixed with those of libwedge.so."""
    global _lib_debug
    if _lib_debug is None:
        path = os.path.join(os.path.dirname(_SO), "libwedge_debug.so")
        if not os.path.exists(path):
            raise ImportError(f"libwedge_debug.so is not built ({path}); run __graft_entry__.build()")
        _lib_debug = _configure(ctypes.CDLL(path))
    return _lib_debug


def _configure(lib):
    """Argument and result types of every exported function; ABI struct sizes checked."""
    i32, i64, u32, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    P = ctypes.c_void_p
    st = ctypes.c_int
    sig = {
        "wedge_status_str": ([st], ctypes.c_char_p),
        "wedge_last_error": ([], ctypes.c_char_p),
        "wedge_version": ([], u32),
        "wedge_abi_sizes": ([P, ctypes.c_int], ctypes.c_int),
        "wedge_graph_build": ([P, P, i64, i32, P, P], st),
        "wedge_graph_free": ([P], None),
        "wedge_graph_get_info": ([P, P], st),
        "wedge_graph_copy": ([P, P, P, P, P], st),
        "wedge_bin": ([P, P, P, P], st),
        "wedge_bins_free": ([P], None),
        "wedge_bins_get_info": ([P, P], st),
        "wedge_bins_copy": ([P, P, P, P], st),
        "wedge_sample": ([P, P, P, P, P], st),
        "wedge_hoeffding_k": ([dbl, dbl], u64),
        "wedge_estimate": ([P, dbl, P], st),
        "wedge_classify": ([P, P, i64, P, P, P, P, P], st),
        "wedge_profile_enable": ([ctypes.c_int], None),
        "wedge_profile_reset": ([], None),
        "wedge_profile_read": ([P, ctypes.c_int], ctypes.c_int),
        "wedge_trim": ([], st),
        "wedge_degree_offsets_noalloc": ([P, i64, P, P], st),
        "wedge_batch_create": ([P, ctypes.c_int, P, P, P], st),
        "wedge_batch_launch": ([P, P], st),
        "wedge_batch_results": ([P, P], st),
        "wedge_batch_free": ([P], None),
        "wedge_batch_info": ([P, P, P, P], st),
        "wedge_sample_batch": ([P, ctypes.c_int, P, P, P], st),
        "wedge_autotune": ([P, ctypes.c_int, P, P], st),
        "wedge_server_create": ([P, P], st),
        "wedge_server_destroy": ([P], None),
        "wedge_server_add_graph": ([P, P, P, i64, i32, P], st),
        "wedge_server_remove_graph": ([P, u64], st),
        "wedge_server_submit": ([P, P, P], st),
        "wedge_server_wait": ([P, u64, P, P], st),
        "wedge_server_stats": ([P, P, ctypes.c_int], st),
        "wedge_probe_random_read": ([u64, u64, P, P], st),
        "wedge_triangle_stats": ([P, P, u64, u64, P, P, P], st),
        "wedge_exact": ([P, P, P, P, P], st),
        "wedge_pool_used_bytes": ([], u64),
        "wedge_test_fail_allocation": ([i64], None),
        "wedge_test_lookback_timeout": ([u32, P], st),
        "wedge_graph_from_csr": ([P, P, i32, i64, P, P], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    sizes = (ctypes.c_uint64 * 32)()
    lib.wedge_abi_sizes(sizes, 32)
    for i, S in enumerate(_STRUCTS):
        if sizes[i] != ctypes.sizeof(S):
            raise ImportError(f"ABI mismatch for {S.__name__}: C {sizes[i]} bytes, binding {ctypes.sizeof(S)}")
    return lib


def _check(status: int):
    if status != 0:
        raise WedgeError(status, _lib.wedge_last_error().decode())


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(a, dtype=None):
    """(pointer, keepalive) of a contiguous torch tensor or numpy array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if dtype is not None:
                want = {np.int32: torch.int32, np.uint8: torch.uint8, np.int64: torch.int64}[dtype]
                if a.dtype != want:
                    raise TypeError(f"expected {want}, got {a.dtype}")
            a = a.contiguous()
            return a.data_ptr(), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype) if dtype is not None else np.ascontiguousarray(a)
    return arr.ctypes.data, arr


# ---------------------------------------------------------------------------
# Handles
# ---------------------------------------------------------------------------

class Graph:
    """Owns a wedge_graph handle (device CSR)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> GraphInfo:
        gi = GraphInfo()
        _check(load().wedge_graph_get_info(self._h, ctypes.byref(gi)))
        return gi

    def copy(self, off=None, adj=None, deg=None, stream=None):
        """Copy the CSR into caller arrays (host or device)."""
        po = _ptr(off, np.int64)[0] if off is not None else 0
        pa = _ptr(adj, np.int32)[0] if adj is not None else 0
        pd = _ptr(deg, np.int32)[0] if deg is not None else 0
        _check(load().wedge_graph_copy(self._h, po, pa, pd, _stream_handle(stream)))

    def csr_numpy(self):
        gi = self.info()
        off = np.empty(gi.n_vertices + 1, np.int64)
        adj = np.empty(max(gi.n_adj, 1), np.int32)
        deg = np.empty(gi.n_vertices, np.int32)
        self.copy(off, adj, deg)
        return off, adj[: gi.n_adj], deg

    def free(self):
        if self._h:
            load().wedge_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Bins:
    """Owns a wedge_bins handle (bin table, L and W on the device)."""

    def __init__(self, handle, graph: Graph):
        self._h = handle
        self.graph = graph

    @property
    def handle(self):
        return self._h

    def info(self) -> BinsInfo:
        bi = BinsInfo()
        _check(load().wedge_bins_get_info(self._h, ctypes.byref(bi)))
        return bi

    def copy(self, L=None, W=None, stream=None):
        """Copy L (int32) and W (uint64, passed as an int64 or uint64 array) into caller arrays."""
        pl = _ptr(L, np.int32)[0] if L is not None else 0
        pw = _ptr(W)[0] if W is not None else 0
        _check(load().wedge_bins_copy(self._h, pl, pw, _stream_handle(stream)))

    def arrays_numpy(self):
        bi = self.info()
        L = np.empty(max(bi.n_wedge_vertices, 1), np.int32)
        W = np.empty(bi.n_wedge_vertices + 1, np.uint64)
        self.copy(L, W)
        return L[: bi.n_wedge_vertices], W

    def free(self):
        if self._h:
            load().wedge_bins_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def graph_build(src, dst, n_vertices: int, stream=None) -> Graph:
    lib = load()
    ps, ks = _ptr(src, np.int32)
    pd, kd = _ptr(dst, np.int32)
    n_edges = int(ks.shape[0]) if hasattr(ks, "shape") else len(ks)
    h = ctypes.c_void_p()
    _check(lib.wedge_graph_build(ps, pd, n_edges, int(n_vertices), _stream_handle(stream), ctypes.byref(h)))
    return Graph(h.value)


def bin(graph: Graph, tau: int = 1, omega: int = 2, stream=None) -> Bins:  # noqa: A001 - C name
    lib = load()
    bp = BinParams(tau, omega)
    h = ctypes.c_void_p()
    _check(lib.wedge_bin(graph.handle, ctypes.byref(bp), _stream_handle(stream), ctypes.byref(h)))
    return Bins(h.value, graph)


class Counts:
    """Host copy of wedge_counts as numpy arrays."""

    def __init__(self, c: CountsStruct):
        self.raw = c
        nb = c.n_bins
        self.n_bins = nb
        self.k_b = np.array(c.k_b[:nb], np.uint64)
        self.q = np.array([list(c.q[i]) for i in range(nb)], np.uint64).reshape(nb, 4)
        self.n_b = np.array(c.n_b[:nb], np.uint64)
        self.p_b = np.array(c.p_b[:nb], np.uint64)
        self.p_total = int(c.p_total)
        self.k_global = int(c.k_global)
        self.closed_global = int(c.closed_global)
        self.stats = np.array([list(c.stats[i]) for i in range(STAT_BINS)], np.uint64)

    def counts_matrix(self):
        """(n_bins, 5) = (k_b, q0, q1, q2, q3), the oracle's layout."""
        return np.concatenate([self.k_b[:, None], self.q], axis=1)


def _budget_array(k_bin):
    if k_bin is None:
        return None
    return np.ascontiguousarray(np.asarray(k_bin, dtype=np.uint64))


def sample(graph: Graph, bins: Bins, seed: int, eps: float = 0.0, delta: float = 0.0, k_per_bin: int = 0,
           k_global: int = 0, flags: int = 0, records=None, stream=None, k_bin=None, first_sample: int = 0) -> Counts:
    """k_bin: optional per-bin budgets indexed by bin id (length >= n_bins);
    first_sample: first sample index of every stream (for sharding)."""
    lib = load()
    kb = _budget_array(k_bin)
    if kb is not None and kb.shape[0] < bins.info().n_bins:
        raise ValueError("k_bin needs one entry per bin id")
    sp = SampleParams(seed, eps, delta, k_per_bin, k_global, flags, _ptr(records)[0] if records is not None else 0,
                      kb.ctypes.data if kb is not None else 0, first_sample)
    c = CountsStruct()
    _check(lib.wedge_sample(graph.handle, bins.handle, ctypes.byref(sp), _stream_handle(stream), ctypes.byref(c)))
    return Counts(c)


def estimate(counts: Counts, delta: float) -> dict:
    lib = load()
    e = EstimatesStruct()
    _check(lib.wedge_estimate(ctypes.byref(counts.raw), delta, ctypes.byref(e)))
    nb = e.n_bins
    return {"c_b": list(e.c_b[:nb]), "t_b": list(e.t_b[:nb]), "eps_b": list(e.eps_b[:nb]), "p": e.p_total,
            "c_hat": e.c_hat, "t_hat": e.t_hat, "c_hat_global": e.c_hat_global, "t_hat_global": e.t_hat_global,
            "eps_global": e.eps_global}


def classify(graph: Graph, bins: Bins, v0, v1, v2, q, stream=None):
    """Closure + class of given wedges (device arrays) into q (device uint8)."""
    lib = load()
    p0, k0 = _ptr(v0, np.int32)
    p1, _ = _ptr(v1, np.int32)
    p2, _ = _ptr(v2, np.int32)
    pq, _ = _ptr(q, np.uint8)
    n = int(k0.shape[0])
    _check(lib.wedge_classify(graph.handle, bins.handle, n, p0, p1, p2, pq, _stream_handle(stream)))


def exact(graph: Graph, bins: Bins, t_i=None, stream=None) -> dict:
    """Exact triangle counts (wedge_exact): t, p_b, pbq[n_bins, 4] (q = 0 open,
    1..3 closed by class); t_i: optional device uint64 tensor of n_vertices."""
    lib = load()
    out = ExactCounts()
    pt = 0
    if t_i is not None:
        pt, arr = _ptr(t_i)
        if int(np.prod(arr.shape)) < graph.info().n_vertices:
            raise ValueError("t_i needs n_vertices entries")
    _check(lib.wedge_exact(graph.handle, bins.handle, pt, _stream_handle(stream), ctypes.byref(out)))
    nb = out.n_bins
    pbq = np.array([list(out.pbq[i]) for i in range(nb)], np.uint64).reshape(nb, 4)
    return {"triangles": int(out.triangles), "p_total": int(out.p_total), "p_b": np.array(out.p_b[:nb], np.uint64),
            "pbq": pbq}


BOX_FIELDS = ("count", "min", "q1", "median", "q3", "max", "whisker_lo", "whisker_hi", "outliers")


def triangle_stats(graph: Graph, bins: Bins, seed: int, k: int, records=None, stream=None) -> dict:
    """Sampled-triangle statistics (wedge_triangle_stats): k global-stream
    samples; "box" is (34, 9) uint64 with columns BOX_FIELDS per BinId(d_min),
    "ratio_q" the min, q1, median, q3, max of d_max / d_min, "hist" the
    (BinId(d_min), BinId(d_max)) histogram. records: optional device buffer of
    k * 8 int32 to receive the per-sample records."""
    lib = load()
    out = TriangleSummary()
    pr = 0
    if records is not None:
        pr, arr = _ptr(records, np.int32)
        if int(np.prod(arr.shape)) < 8 * k:
            raise ValueError("records needs k * 8 int32 entries")
    _check(lib.wedge_triangle_stats(graph.handle, bins.handle, seed, k, pr, _stream_handle(stream),
                                    ctypes.byref(out)))
    box = np.array([[getattr(out.box[i], f) for f in BOX_FIELDS] for i in range(STAT_BINS)], np.uint64)
    return {"k": int(out.k), "closed": int(out.closed), "box": box, "ratio_q": np.array(out.ratio_q[:], np.float64),
            "hist": np.array([list(out.hist[i]) for i in range(STAT_BINS)], np.uint64)}


NOALLOC_MAX_VERTICES = 536870912


def degree_offsets_noalloc(deg, off, stream=None):
    """Row offsets off[0..n] from device degrees deg[0..n) without any device
    allocation (wedge_degree_offsets_noalloc). deg: contiguous int32 CUDA
    tensor; off: contiguous int64 CUDA tensor of at least n + 1 entries, on
    the same (current) device, written in place."""
    import torch
    lib = load()
    for name, t, dt in (("deg", deg, torch.int32), ("off", off, torch.int64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous (off is written in place)")
    n = deg.numel()
    if off.numel() < n + 1:
        raise ValueError(f"off holds {off.numel()} entries; n + 1 = {n + 1} are needed")
    _check(lib.wedge_degree_offsets_noalloc(deg.data_ptr(), n, off.data_ptr(), _stream_handle(stream)))


def pool_used_bytes() -> int:
    """Bytes of the library's device pool currently handed out (current device)."""
    return int(load().wedge_pool_used_bytes())


def fail_next_allocation(after: int):
    """Test hook: refuse the library's device allocation that follows `after`
    more successful ones (WEDGE_ENOMEM); negative disarms."""
    load().wedge_test_fail_allocation(int(after))


def force_lookback_timeout(spin_limit: int, stream=None):
    """Test hook: a scan whose look-back waits on a status word nothing sets,
    with the poll limit lowered to spin_limit; raises WedgeError(ETIMEOUT)."""
    _check(load().wedge_test_lookback_timeout(int(spin_limit), _stream_handle(stream)))


def graph_from_csr(off, adj, n_vertices: int, stream=None) -> "Graph":
    """A graph from a saved CSR (host or device arrays; wedge_graph_from_csr)."""
    lib = load()
    po, ko = _ptr(off, np.int64)
    pa, ka = _ptr(adj, np.int32)
    n_adj = int(ka.shape[0]) if hasattr(ka, "shape") else int(ka.numel())
    if int(ko.shape[0]) != int(n_vertices) + 1:
        raise ValueError("off must hold n_vertices + 1 entries")
    h = ctypes.c_void_p()
    _check(lib.wedge_graph_from_csr(po, pa if n_adj else None, int(n_vertices), n_adj, _stream_handle(stream),
                                    ctypes.byref(h)))
    return Graph(h.value)


def graph_save(graph: "Graph", path: str):
    """Save a graph's CSR to a .npz file (checkpoint; reload with graph_load)."""
    off, adj, _ = graph.csr_numpy()
    np.savez(path, off=off, adj=adj, n_vertices=np.int64(off.shape[0] - 1))


def graph_load(path: str, stream=None) -> "Graph":
    """A graph from a file written by graph_save (validated on the device)."""
    z = np.load(path)
    return graph_from_csr(z["off"], z["adj"], int(z["n_vertices"]), stream=stream)


def hoeffding_k(eps: float, delta: float) -> int:
    return int(load().wedge_hoeffding_k(eps, delta))


def profile_enable(timing: bool = True):
    load().wedge_profile_enable(1 if timing else 0)


def profile_reset():
    load().wedge_profile_reset()


def profile_read() -> dict:
    lib = load()
    n = lib.wedge_profile_read(None, 0)
    arr = (KernelStat * max(n, 1))()
    n = lib.wedge_profile_read(arr, n)
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms),
                                   "first_start_ms": float(arr[i].first_start_ms),
                                   "last_end_ms": float(arr[i].last_end_ms)}
            for i in range(n)}


def probe_random_read(buffer_bytes: int = 32 << 30, reads: int = 1 << 30, stream=None) -> float:
    """Random 32-byte sector reads per second (wedge_probe_random_read)."""
    r = ctypes.c_double()
    _check(load().wedge_probe_random_read(buffer_bytes, reads, _stream_handle(stream), ctypes.byref(r)))
    return r.value


def trim():
    _check(load().wedge_trim())


# ---------------------------------------------------------------------------
# Batched sampling (wedge_batch_*, wedge_autotune)
# ---------------------------------------------------------------------------

class Requests:
    """A C array of wedge_request plus the host budget arrays it points to."""

    def __init__(self, items):
        """items: iterable of dicts with graph, bins, seed and any of eps, delta,
        k_per_bin, k_global, k_bin, flags, records."""
        items = list(items)
        self.n = len(items)
        self.array = (Request * max(self.n, 1))()
        self._keep = []
        for i, it in enumerate(items):
            kb = _budget_array(it.get("k_bin"))
            if kb is not None:
                self._keep.append(kb)
            rec = it.get("records")
            if rec is not None:
                self._keep.append(rec)
            self.array[i].graph = it["graph"].handle
            self.array[i].bins = it["bins"].handle
            self.array[i].params = SampleParams(it.get("seed", 0), it.get("eps", 0.0), it.get("delta", 0.0),
                                                it.get("k_per_bin", 0), it.get("k_global", 0), it.get("flags", 0),
                                                _ptr(rec)[0] if rec is not None else 0,
                                                kb.ctypes.data if kb is not None else 0, it.get("first_sample", 0))
        self.items = items


def _config(cfg):
    if cfg is None:
        return None
    if isinstance(cfg, LaunchConfig):
        return cfg
    c = LaunchConfig()
    for k, v in cfg.items():
        setattr(c, k, int(v))
    return c


class Batch:
    """A planned batch (one descriptor per stream on the device, CUDA-graph-captured launch)."""

    def __init__(self, requests: Requests, cfg=None, stream=None):
        lib = load()
        self.requests = requests
        c = _config(cfg)
        h = ctypes.c_void_p()
        _check(lib.wedge_batch_create(requests.array, requests.n, ctypes.byref(c) if c is not None else None,
                                      _stream_handle(stream), ctypes.byref(h)))
        self._h = h.value

    def info(self):
        ns, nt, gr = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(load().wedge_batch_info(self._h, ctypes.byref(ns), ctypes.byref(nt), ctypes.byref(gr)))
        return {"streams": ns.value, "tiles": nt.value, "grid": gr.value}

    def launch(self, stream=None):
        _check(load().wedge_batch_launch(self._h, _stream_handle(stream)))

    def results(self):
        out = (CountsStruct * max(self.requests.n, 1))()
        _check(load().wedge_batch_results(self._h, out))
        return [Counts(out[i]) for i in range(self.requests.n)]

    def free(self):
        if self._h:
            load().wedge_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sample_batch(requests: Requests, cfg=None, stream=None):
    """All requests in one persistent launch (wedge_sample_batch)."""
    lib = load()
    c = _config(cfg)
    out = (CountsStruct * max(requests.n, 1))()
    _check(lib.wedge_sample_batch(requests.array, requests.n, ctypes.byref(c) if c is not None else None,
                                  _stream_handle(stream), out))
    return [Counts(out[i]) for i in range(requests.n)]


def autotune(requests: Requests, stream=None) -> LaunchConfig:
    lib = load()
    c = LaunchConfig()
    _check(lib.wedge_autotune(requests.array, requests.n, _stream_handle(stream), ctypes.byref(c)))
    return c


# ---------------------------------------------------------------------------
# Serving (wedge_server_*)
# ---------------------------------------------------------------------------

class Server:
    """Continuous-batching request loop over resident graphs."""

    def __init__(self, hbm_budget_bytes: int = 0, slots: int = 2, max_batch_requests: int = 0, tau: int = 1,
                 omega: int = 2, launch=None, max_batch_samples: int = 0, max_queued_samples: int = 0,
                 gpu_filling_samples: int = 0):
        lib = load()
        c = ServerConfig()
        c.hbm_budget_bytes = int(hbm_budget_bytes)
        c.slots = int(slots)
        c.max_batch_requests = int(max_batch_requests)
        c.tau = int(tau)
        c.omega = int(omega)
        c.max_batch_samples = int(max_batch_samples)
        c.max_queued_samples = int(max_queued_samples)
        c.gpu_filling_samples = int(gpu_filling_samples)
        lc = _config(launch)
        if lc is not None:
            c.launch = lc
        h = ctypes.c_void_p()
        _check(lib.wedge_server_create(ctypes.byref(c), ctypes.byref(h)))
        self._h = h.value

    def add_graph(self, src, dst, n_vertices: int) -> int:
        ps, ks = _ptr(src, np.int32)
        pd, _ = _ptr(dst, np.int32)
        gid = ctypes.c_uint64()
        _check(load().wedge_server_add_graph(self._h, ps, pd, int(ks.shape[0]), int(n_vertices), ctypes.byref(gid)))
        return gid.value

    def remove_graph(self, graph_id: int):
        _check(load().wedge_server_remove_graph(self._h, graph_id))

    def submit(self, graph_id: int, seed: int, eps: float = 0.0, delta: float = 0.0, k_per_bin: int = 0,
               k_global: int = 0, flags: int = 0) -> int:
        r = ServerRequest(graph_id, seed, eps, delta, k_per_bin, k_global, flags, 0)
        t = ctypes.c_uint64()
        _check(load().wedge_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int):
        c = CountsStruct()
        tm = RequestTiming()
        _check(load().wedge_server_wait(self._h, ticket, ctypes.byref(c), ctypes.byref(tm)))
        return Counts(c), {"submit_us": tm.submit_us, "dispatch_us": tm.dispatch_us, "done_us": tm.done_us,
                           "latency_us": tm.done_us - tm.submit_us, "batch_requests": tm.batch_requests}

    def stats(self, reset: bool = False) -> dict:
        m = ServerMetrics()
        _check(load().wedge_server_stats(self._h, ctypes.byref(m), 1 if reset else 0))
        return {f: (getattr(m, f) if not isinstance(getattr(m, f), int) else int(getattr(m, f)))
                for f, _ in m._fields_ if f != "reserved"}

    def close(self):
        if self._h:
            load().wedge_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
