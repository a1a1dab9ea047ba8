"""GPU path vs the CPU oracle, through the C ABI (needs a GB300).

Integer results (CSR, bins, L, W, per-bin tallies, global counts, statistics
histogram, per-sample records) must match the oracle bit for bit; FP64
estimates within 1e-12 relative.
"""
import math
from itertools import combinations

import numpy as np
import pytest

import graphgen
import oracle
from oracle import brute
from oracle.estimate import estimate as oracle_estimate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
wedge = pytest.importorskip("paper_1301_5887_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    wedge.load()


def dev(a, dtype=torch.int32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def check_csr(g, src, dst, n):
    off, adj = oracle.csr(src, dst, n)
    goff, gadj, gdeg = g.csr_numpy()
    assert np.array_equal(goff, off)
    assert np.array_equal(gadj, adj)
    assert np.array_equal(gdeg, np.diff(off).astype(np.int32))
    gi = g.info()
    assert gi.n_adj == adj.shape[0]
    assert gi.max_degree == (int(np.diff(off).max()) if n > 0 and adj.shape[0] else 0)
    return off, adj


def oracle_L_W(off, tau, omega):
    d = np.diff(off)
    bins_of = np.array([oracle.bin_id(int(x), tau, omega) for x in d], np.int64)
    ids = np.nonzero(d >= 2)[0]
    order = np.lexsort((ids, bins_of[ids]))
    L = ids[order].astype(np.int32)
    w = (d[L].astype(np.uint64) * (d[L].astype(np.uint64) - np.uint64(1))) // np.uint64(2)
    W = np.concatenate([[np.uint64(0)], np.cumsum(w, dtype=np.uint64)])
    return L, W


def check_bins(b, off, tau, omega):
    ref = oracle.bins(off, tau, omega)
    bi = b.info()
    nb = ref["n_bins"]
    assert bi.n_bins == nb
    assert list(bi.n_b[:nb]) == [int(x) for x in ref["n_b"]]
    assert list(bi.p_b[:nb]) == [int(x) for x in ref["p_b"]]
    assert list(bi.lo_deg[:nb]) == [int(x) for x in ref["lo"]]
    assert bi.p_total == int(ref["p_b"].sum())
    L, W = oracle_L_W(off, tau, omega)
    assert bi.n_wedge_vertices == L.shape[0]
    gL, gW = b.arrays_numpy()
    assert np.array_equal(gL, L)
    assert np.array_equal(gW, W)
    return ref


def check_counts(c, ref):
    nb = ref["counts"].shape[0]
    assert c.n_bins == nb
    assert np.array_equal(c.counts_matrix(), ref["counts"])
    assert c.k_global == int(ref["glob"][0])
    assert c.closed_global == int(ref["glob"][1])
    assert np.array_equal(c.stats, ref["stats"])


def check_estimates(c, ref, p_b, delta):
    got = wedge.estimate(c, delta)
    exp = oracle_estimate(p_b, ref["counts"], ref["glob"], delta)
    for key in ["c_hat", "t_hat", "c_hat_global", "t_hat_global"]:
        assert got[key] == pytest.approx(exp[key], rel=1e-12, abs=1e-300)
    for b in range(len(exp["c_b"])):
        assert got["c_b"][b] == pytest.approx(exp["c_b"][b], rel=1e-12, abs=1e-300)
        assert got["t_b"][b] == pytest.approx(exp["t_b"][b], rel=1e-12, abs=1e-300)
    return got


# ---------------------------------------------------------------------------
# Worked example and small graphs
# ---------------------------------------------------------------------------

def test_fig_example_end_to_end():
    e = np.array([[0, 1], [0, 2], [1, 3], [2, 3], [2, 4], [3, 4], [3, 5]], np.int32)
    g = wedge.graph_build(e[:, 0], e[:, 1], 6)  # host input
    off, adj = check_csr(g, e[:, 0], e[:, 1], 6)
    b = wedge.bin(g, tau=10, omega=2)
    check_bins(b, off, 10, 2)
    rec = torch.zeros((3000, 8), dtype=torch.int32, device="cuda")
    c = wedge.sample(g, b, seed=3, k_per_bin=1000, k_global=3000, records=rec)
    ref = oracle.sample(off, adj, 10, 2, 3, 1000, 3000, records=True)
    check_counts(c, ref)
    assert np.array_equal(rec.cpu().numpy(), ref["records"])


def test_classify_exhaustive_equals_oracle_and_exact():
    src, dst = graphgen.kronecker_host(8)
    g = wedge.graph_build(dev(src), dev(dst), 256)
    off, adj = check_csr(g, src, dst, 256)
    for tau, omega in [(1, 2), (2, 2), (4, 3)]:
        b = wedge.bin(g, tau=tau, omega=omega)
        v0, v1, v2 = [], [], []
        for cc in range(256):
            for i, j in combinations(adj[off[cc]:off[cc + 1]].tolist(), 2):
                v0.append(cc), v1.append(i), v2.append(j)
        q = torch.zeros(len(v0), dtype=torch.uint8, device="cuda")
        wedge.classify(g, b, dev(v0), dev(v1), dev(v2), q)
        qg = q.cpu().numpy()
        assert np.array_equal(qg, oracle.classify(off, adj, tau, omega, v0, v1, v2))
        ex = oracle.exact(off, adj, tau, omega)
        d = np.diff(off)
        pbq = np.zeros_like(ex["pbq"])
        for cc, qq in zip(v0, qg.tolist()):
            pbq[oracle.bin_id(int(d[cc]), tau, omega), qq] += 1
        assert np.array_equal(pbq, ex["pbq"])


def test_classify_rejects_bad_ids():
    src, dst = graphgen.kronecker_host(6)
    g = wedge.graph_build(dev(src), dev(dst), 64)
    b = wedge.bin(g)
    q = torch.zeros(2, dtype=torch.uint8, device="cuda")
    with pytest.raises(wedge.WedgeError) as e:
        wedge.classify(g, b, dev([0, 64]), dev([1, 2]), dev([2, 3]), q)
    assert e.value.status == 1


@pytest.mark.parametrize("n,m,seed,on_device", [(50, 40, 0, True), (300, 2000, 1, False), (1000, 30000, 2, True),
                                                (5000, 4097, 3, True), (70000, 65537, 4, False)])
def test_random_multigraph_csr(n, m, seed, on_device):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    # duplicates, reversed pairs and self-loops
    src = np.concatenate([src, dst[: m // 3], src[: m // 5], np.arange(min(n, 7), dtype=np.int32)])
    dst = np.concatenate([dst, src[: m // 3], dst[: m // 5], np.arange(min(n, 7), dtype=np.int32)])
    g = wedge.graph_build(dev(src) if on_device else src, dev(dst) if on_device else dst, n)
    check_csr(g, src, dst, n)


@pytest.mark.parametrize("m", [1, 2, 31, 2047, 2048, 2049, 4095, 4096, 4097, 12289])
def test_ragged_edge_counts(m):
    rng = np.random.default_rng(m)
    n = 3000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    g = wedge.graph_build(dev(src), dev(dst), n)
    off, adj = check_csr(g, src, dst, n)
    b = wedge.bin(g, tau=1, omega=2)
    check_bins(b, off, 1, 2)
    c = wedge.sample(g, b, seed=m, k_per_bin=777, k_global=2049)
    check_counts(c, oracle.sample(off, adj, 1, 2, m, 777, 2049))


def test_heavy_duplicates_across_tiles():
    """Long runs of one key straddle sort, dedup and scan tiles."""
    n = 100
    src = np.repeat(np.arange(10, dtype=np.int32), 5000)
    dst = np.tile(np.arange(50, 60, dtype=np.int32), 5000)
    g = wedge.graph_build(dev(src), dev(dst), n)
    check_csr(g, src, dst, n)


# ---------------------------------------------------------------------------
# Kronecker workloads
# ---------------------------------------------------------------------------

def test_device_generator_matches_host():
    for scale in [5, 12, 13]:
        m = graphgen.kronecker_edges(scale)
        s = torch.empty(m, dtype=torch.int32, device="cuda")
        d = torch.empty(m, dtype=torch.int32, device="cuda")
        graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), m, torch.cuda.current_stream().cuda_stream)
        hs, hd = graphgen.kronecker_host(scale)
        assert np.array_equal(s.cpu().numpy(), hs) and np.array_equal(d.cpu().numpy(), hd)


def _device_kronecker(scale):
    m = graphgen.kronecker_edges(scale)
    s = torch.empty(m, dtype=torch.int32, device="cuda")
    d = torch.empty(m, dtype=torch.int32, device="cuda")
    graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), m, torch.cuda.current_stream().cuda_stream)
    return s, d


def test_kronecker_scale12_config():
    """Scale 12, edge factor 16, permuted ids, bins 2^i <= d < 2^(i+1),
    10,000 samples per nonempty bin and 100,000 global, Philox seed 7."""
    s, d = _device_kronecker(12)
    g = wedge.graph_build(s, d, 4096)
    hs, hd = graphgen.kronecker_host(12)
    off, adj = check_csr(g, hs, hd, 4096)
    b = wedge.bin(g, tau=1, omega=2)
    ref_bins = check_bins(b, off, 1, 2)
    rec = torch.zeros((100000, 8), dtype=torch.int32, device="cuda")
    c = wedge.sample(g, b, seed=7, k_per_bin=10000, k_global=100000, records=rec)
    ref = oracle.sample(off, adj, 1, 2, 7, 10000, 100000, records=True)
    check_counts(c, ref)
    assert np.array_equal(rec.cpu().numpy(), ref["records"])
    est = check_estimates(c, ref, ref_bins["p_b"], 0.001)
    # against brute-force exact counts: within the Hoeffding half-width of each bin
    ex = oracle.exact(off, adj, 1, 2)
    for bb in range(ref_bins["n_bins"]):
        pb = int(ex["p_b"][bb])
        if pb == 0:
            continue
        pbq = [int(x) for x in ex["pbq"][bb]]
        assert abs(est["c_b"][bb] - (pbq[1] + pbq[2] + pbq[3]) / pb) < est["eps_b"][bb]
    assert abs(est["c_hat_global"] - 3 * ex["t"] / int(ex["p_b"].sum())) < est["eps_global"]


@pytest.mark.parametrize("tau,omega", [(2, 2), (3, 3), (1, 10**7), (5, 7), (40, 2)])
def test_general_bins(tau, omega):
    s, d = _device_kronecker(11)
    g = wedge.graph_build(s, d, 2048)
    hs, hd = graphgen.kronecker_host(11)
    off, adj = check_csr(g, hs, hd, 2048)
    b = wedge.bin(g, tau=tau, omega=omega)
    check_bins(b, off, tau, omega)
    c = wedge.sample(g, b, seed=11, k_per_bin=3000, k_global=5000)
    check_counts(c, oracle.sample(off, adj, tau, omega, 11, 3000, 5000))


def test_budget_from_eps_delta_and_flags():
    s, d = _device_kronecker(10)
    g = wedge.graph_build(s, d, 1024)
    hs, hd = graphgen.kronecker_host(10)
    off, adj = oracle.csr(hs, hd, 1024)
    b = wedge.bin(g)
    k = oracle.hoeffding_k(0.05, 0.01)
    c = wedge.sample(g, b, seed=5, eps=0.05, delta=0.01)
    check_counts(c, oracle.sample(off, adj, 1, 2, 5, k, k))
    c2 = wedge.sample(g, b, seed=5, k_per_bin=100, k_global=100, flags=wedge.FLAG_NO_GLOBAL)
    assert c2.k_global == 0 and c2.closed_global == 0 and int(c2.k_b.sum()) > 0
    c3 = wedge.sample(g, b, seed=5, k_per_bin=100, k_global=100, flags=wedge.FLAG_NO_BINS)
    assert int(c3.k_b.sum()) == 0 and c3.k_global == 100
    ref = oracle.sample(off, adj, 1, 2, 5, 100, 100)
    assert c3.closed_global == int(ref["glob"][1])


def test_repeatable_and_stream_independent():
    s, d = _device_kronecker(11)
    g = wedge.graph_build(s, d, 2048)
    b = wedge.bin(g)
    a = wedge.sample(g, b, seed=99, k_per_bin=5000, k_global=5000)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        c = wedge.sample(g, b, seed=99, k_per_bin=5000, k_global=5000, stream=side)
    assert np.array_equal(a.counts_matrix(), c.counts_matrix()) and a.closed_global == c.closed_global


# ---------------------------------------------------------------------------
# Edge cases and errors
# ---------------------------------------------------------------------------

def test_empty_and_degenerate_graphs():
    for src, dst, n in [([], [], 5), ([3, 3, 3], [3, 3, 3], 5), ([0], [1], 2), ([0], [0], 1)]:
        src = np.array(src, np.int32)
        dst = np.array(dst, np.int32)
        g = wedge.graph_build(src, dst, n)
        off, adj = check_csr(g, src, dst, n)
        b = wedge.bin(g)
        bi = b.info()
        assert bi.p_total == 0 and bi.n_wedge_vertices == 0
        c = wedge.sample(g, b, seed=1, k_per_bin=10, k_global=10)
        assert int(c.k_b.sum()) == 0 and c.k_global == 0


def test_build_errors():
    with pytest.raises(wedge.WedgeError) as e:
        wedge.graph_build(np.array([0, 5], np.int32), np.array([1, 1], np.int32), 5)
    assert e.value.status == 1
    with pytest.raises(wedge.WedgeError) as e:
        wedge.graph_build(dev([0, -1]), dev([1, 1]), 5)
    assert e.value.status == 1
    with pytest.raises(wedge.WedgeError):
        wedge.graph_build(np.array([0], np.int32), np.array([0], np.int32), 0)
    # the library keeps working after errors
    g = wedge.graph_build(np.array([0, 1], np.int32), np.array([1, 2], np.int32), 3)
    assert g.info().n_adj == 4


def test_bin_and_sample_errors():
    src, dst = graphgen.kronecker_host(9)
    g = wedge.graph_build(dev(src), dev(dst), 512)
    g2 = wedge.graph_build(dev(src), dev(dst), 512)
    for tau, omega in [(0, 2), (1, 1), (1, 2**33)]:
        with pytest.raises(wedge.WedgeError) as e:
            wedge.bin(g, tau=tau, omega=omega)
        assert e.value.status == 1
    star = wedge.graph_build(np.zeros(400, np.int32), np.arange(1, 401, dtype=np.int32), 401)
    with pytest.raises(wedge.WedgeError) as e:  # singleton bins up to degree 400 exceed the bin table
        wedge.bin(star, tau=1000, omega=2)
    assert e.value.status == 1
    b = wedge.bin(g)
    with pytest.raises(wedge.WedgeError):
        wedge.sample(g2, b, seed=1, k_per_bin=10, k_global=10)
    with pytest.raises(wedge.WedgeError):
        wedge.sample(g, b, seed=1, eps=0.0, delta=0.1)
    rec = torch.zeros((10, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(wedge.WedgeError):
        wedge.sample(g, b, seed=1, k_per_bin=10, k_global=10, flags=wedge.FLAG_NO_GLOBAL, records=rec)


def test_maximum_vertex_ids():
    """n = 2^31 - 1: 31-bit ids, 62-bit keys (eight radix passes)."""
    n = 2**31 - 1
    rng = np.random.default_rng(5)
    pool = np.array([0, 1, 2, n - 1, n - 2, n - 3, 2**30, 2**30 + 1], np.int64)
    pool = np.concatenate([pool, rng.integers(0, n, 40)])
    src = rng.choice(pool, 3000).astype(np.int32)
    dst = rng.choice(pool, 3000).astype(np.int32)
    g = wedge.graph_build(dev(src), dev(dst), n)
    gi = g.info()
    E = brute.edge_set(src, dst)
    assert gi.n_adj == 2 * len(E)
    verts = np.unique(pool).astype(np.int64)
    off_full = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    g.copy(off=off_full)
    adj = torch.empty(gi.n_adj, dtype=torch.int32, device="cuda")
    g.copy(adj=adj)
    idx = torch.as_tensor(verts).cuda()
    starts = off_full[idx].cpu().numpy()
    ends = off_full[idx + 1].cpu().numpy()
    adj_h = adj.cpu().numpy()
    rows = {}
    for e in E:
        u, v = tuple(e)
        rows.setdefault(u, set()).add(v)
        rows.setdefault(v, set()).add(u)
    for v, a, z in zip(verts.tolist(), starts.tolist(), ends.tolist()):
        assert adj_h[a:z].tolist() == sorted(rows.get(v, set()))
    assert int(off_full[-1].item()) == gi.n_adj
    del off_full
    b = wedge.bin(g)
    assert b.info().n_wedge_vertices == sum(1 for v in rows if len(rows[v]) >= 2)


def test_host_input_streams_in_chunks():
    """A host edge list crosses the link in groups of at most an eighth of it,
    each sorted on its own, and the sorted groups are merged pairwise; pinned
    and pageable host input give the device-input CSR bit for bit."""
    n = 1 << 22
    m = 80_000_001  # groups of 2^24 edges: four full ones and a ragged fifth
    hs, hd = graphgen.kronecker_host(22, n_edges=m, seed=5)
    ref = wedge.graph_build(torch.as_tensor(hs).cuda(), torch.as_tensor(hd).cuda(), n).csr_numpy()
    for src, dst in ((hs, hd), (torch.as_tensor(hs).pin_memory(), torch.as_tensor(hd).pin_memory())):
        got = wedge.graph_build(src, dst, n).csr_numpy()
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
    wedge.profile_reset()
    wedge.profile_enable(False)
    wedge.graph_build(hs, hd, n)
    prof = wedge.profile_read()
    assert prof["edge_histograms"]["launches"] == 5  # one per group; the first sort pass reads the edges
    # 5 sorted groups merged pairwise in a binary tree, each merge queued once
    # its last group is sorted: 3 merges (one a copy of the unpaired run) at
    # level 1, 2 at level 2, 1 at level 3
    assert prof["merge_runs"]["launches"] == 3 + 2 + 1


@pytest.mark.parametrize("m,n", [(4097, 700), (8193, 700), (32768, 700), (32769, 700), (40961, 200),
                                 (65536 * 3 + 5, 700), (50000, 200)])
def test_host_input_group_merge_boundaries(m, n):
    """Two to eight groups, one-key and ragged last groups, unpaired runs in a
    merge pass, odd and even sort pass counts (ids of 10 and 8 bits), and a
    run of repeated keys across groups and merge tiles."""
    rng = np.random.default_rng(m)
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    src[: m // 4] = 3  # one long run of equal keys over several groups and tiles
    dst[: m // 4] = 5
    got = wedge.graph_build(src, dst, n).csr_numpy()
    ref = wedge.graph_build(dev(src), dev(dst), n).csr_numpy()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    check_csr(wedge.graph_build(src, dst, n), src, dst, n)


def test_profile_counts_launches():
    wedge.profile_reset()
    wedge.profile_enable(True)
    s, d = _device_kronecker(10)
    g = wedge.graph_build(s, d, 1024)
    b = wedge.bin(g)
    wedge.sample(g, b, seed=1, k_per_bin=100, k_global=100)
    st = wedge.profile_read()
    wedge.profile_enable(False)
    for name in ["edge_histograms", "sort_onesweep_pass", "dedup_rows", "scan_degrees", "bin_count",
                 "bin_scatter", "sample_closure"]:
        assert st[name]["launches"] >= 1, name
        assert st[name]["total_ms"] > 0.0, name
    # forward keys over 2 x 10 id bits, transposed keys over the larger endpoint's 10 bits
    assert st["sort_onesweep_pass"]["launches"] == math.ceil(2 * 10 / 8) + math.ceil(10 / 8)
    assert "sort_histogram" not in st  # digit histograms come from one pass over the edges
    assert "expand_edges" not in st  # the first sort pass computes the keys from the edges


# ---------------------------------------------------------------------------
# Scale 20 (1,048,576 vertices, 16,777,216 generated edges)
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_kronecker_scale20_config():
    """eps = 0.002, delta = 0.001 -> 950,114 samples per bin and globally:
    bit-exact tallies vs the oracle and estimates within eps of exact counts."""
    scale, n = 20, 1 << 20
    s, d = _device_kronecker(scale)
    g = wedge.graph_build(s, d, n)
    hs, hd = graphgen.kronecker_host(scale)
    off, adj = check_csr(g, hs, hd, n)
    b = wedge.bin(g, tau=1, omega=2)
    ref_bins = check_bins(b, off, 1, 2)
    k = 950114
    c = wedge.sample(g, b, seed=7, k_per_bin=k, k_global=k)
    ref = oracle.sample(off, adj, 1, 2, 7, k, k)
    check_counts(c, ref)
    est = check_estimates(c, ref, ref_bins["p_b"], 0.001)
    ex = oracle.exact(off, adj, 1, 2)
    eps = 0.002
    for bb in range(ref_bins["n_bins"]):
        pb = int(ex["p_b"][bb])
        if pb == 0:
            continue
        pbq = [int(x) for x in ex["pbq"][bb]]
        c_b = (pbq[1] + pbq[2] + pbq[3]) / pb
        t_b = pbq[1] + pbq[2] / 2 + pbq[3] / 3
        assert abs(est["c_b"][bb] - c_b) < eps
        assert abs(est["t_b"][bb] - t_b) < eps * pb
    assert abs(est["c_hat_global"] - 3 * ex["t"] / int(ex["p_b"].sum())) < eps


def test_sharded_sample_ranges_sum_to_full():
    """first_sample shards of every stream sum to the unsharded counts, and
    records of a shard are the matching slice of the full records."""
    from paper_1301_5887_gb300 import multi
    s, d = _device_kronecker(12)
    g = wedge.graph_build(s, d, 4096)
    b = wedge.bin(g)
    k = 30001
    rec_full = torch.zeros((k, 8), dtype=torch.int32, device="cuda")
    full = wedge.sample(g, b, seed=3, k_per_bin=k, k_global=k, records=rec_full)
    tot = np.zeros_like(full.counts_matrix())
    closed = 0
    for r in range(4):
        first, cnt = multi.shard_range(k, r, 4)
        rec = torch.zeros((cnt, 8), dtype=torch.int32, device="cuda")
        c = wedge.sample(g, b, seed=3, k_per_bin=cnt, k_global=cnt, first_sample=first, records=rec)
        tot += c.counts_matrix()
        closed += c.closed_global
        assert torch.equal(rec, rec_full[first:first + cnt])
    assert np.array_equal(tot, full.counts_matrix()) and closed == full.closed_global
