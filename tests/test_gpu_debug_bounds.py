"""The bounds-checked build (libwedge_debug.so, compiled with
-DWEDGE_DEBUG_BOUNDS) on small cases: every index check at a gathered-offset
access (sort scatter and rank positions, the placing pass, dedup, forward
and backward placement, bin scatter, the sampler's gathers) passes, and the
results are the release build's bit for bit. A check that fails records an
error word instead of faulting, and the call returns WEDGE_ECUDA; a clean
run of this file means no index in these paths left its buffer.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
wedge = pytest.importorskip("paper_1301_5887_gb300")


@pytest.fixture(scope="module")
def dbg():
    import __graft_entry__
    __graft_entry__.build()
    wedge.load()
    return wedge.load_debug()


def _ok(lib, st):
    assert st == 0, lib.wedge_last_error().decode()


def _build(lib, src, dst, n):
    h = ctypes.c_void_p()
    ps, _ = wedge._ptr(src, np.int32)
    pd, _ = wedge._ptr(dst, np.int32)
    _ok(lib, lib.wedge_graph_build(ps, pd, int(src.shape[0]), int(n), None, ctypes.byref(h)))
    gi = wedge.GraphInfo()
    _ok(lib, lib.wedge_graph_get_info(h, ctypes.byref(gi)))
    off = np.empty(n + 1, np.int64)
    adj = np.empty(max(gi.n_adj, 1), np.int32)
    _ok(lib, lib.wedge_graph_copy(h, off.ctypes.data, adj.ctypes.data, None, None))
    return h, off, adj[: gi.n_adj]


def _sample(lib, g, seed, k_bin, k_glob, m_records):
    hb = ctypes.c_void_p()
    bp = wedge.BinParams(1, 2)
    _ok(lib, lib.wedge_bin(g, ctypes.byref(bp), None, ctypes.byref(hb)))
    rec = torch.zeros(k_glob * 8, dtype=torch.int32, device="cuda")
    sp = wedge.SampleParams(seed, 0.0, 0.0, k_bin, k_glob, 0, rec.data_ptr(), None, 0)
    c = wedge.CountsStruct()
    _ok(lib, lib.wedge_sample(g, hb, ctypes.byref(sp), None, ctypes.byref(c)))
    counts = np.array([[c.k_b[b]] + list(c.q[b]) for b in range(c.n_bins)], np.uint64)
    out = (counts, int(c.closed_global), np.array([list(r) for r in c.stats], np.uint64), rec.cpu().numpy())
    lib.wedge_bins_free(hb)
    return out


@pytest.mark.parametrize("case", ["kronecker", "multigraph", "host"])
def test_debug_build_matches_release(dbg, case):
    if case == "multigraph":  # duplicates, self-loops, both directions
        rng = np.random.default_rng(3)
        n, m = 3000, 40000
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        src[:500] = dst[:500]
    else:
        src, dst = graphgen.kronecker_host(12, seed=4)
        n = 1 << 12
    if case == "host":
        s_in, d_in = torch.as_tensor(src).pin_memory(), torch.as_tensor(dst).pin_memory()
    else:
        s_in, d_in = torch.as_tensor(src).cuda(), torch.as_tensor(dst).cuda()
    g, off, adj = _build(dbg, s_in, d_in, n)
    ref_off, ref_adj = oracle.csr(src, dst, n)
    assert np.array_equal(off, ref_off) and np.array_equal(adj, ref_adj)
    counts, closed, stats, rec = _sample(dbg, g, 9, 3000, 4000, 4000)
    rg = wedge.graph_build(s_in, d_in, n)
    rb = wedge.bin(rg, tau=1, omega=2)
    rrec = torch.zeros(4000 * 8, dtype=torch.int32, device="cuda")
    rc = wedge.sample(rg, rb, seed=9, k_per_bin=3000, k_global=4000, records=rrec)
    assert np.array_equal(counts, rc.counts_matrix()) and closed == rc.closed_global
    assert np.array_equal(stats, rc.stats)
    assert np.array_equal(rec, rrec.cpu().numpy())
    dbg.wedge_graph_free(g)
    rb.free()
    rg.free()
