"""wedge_exact (Sec. 2.1, 2.2) on GB300 against the oracle's enumeration:
t, p_b and every p_{b,q} identical; t_i identical. At full size (slow):
sampled t_i against neighbour-row intersections the oracle computes one
vertex at a time, and the sampler's per-bin estimates within Hoeffding's
bound of the exact values on a noisy Graph500 graph.
"""
import math
from itertools import combinations

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
wedge = pytest.importorskip("paper_1301_5887_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    wedge.load()


def _check(src, dst, n, tau=1, omega=2, with_ti=True):
    g = wedge.graph_build(src, dst, n)
    b = wedge.bin(g, tau=tau, omega=omega)
    ti = torch.zeros(n, dtype=torch.int64, device="cuda") if with_ti else None
    got = wedge.exact(g, b, t_i=ti)
    off, adj = oracle.csr(src, dst, n)
    ref = oracle.exact(off, adj, tau, omega)
    assert got["triangles"] == ref["t"]
    assert np.array_equal(got["p_b"], ref["p_b"])
    assert np.array_equal(got["pbq"], ref["pbq"])
    if with_ti:
        assert np.array_equal(ti.cpu().numpy().astype(np.uint64), ref["t_i"])
    return got


@pytest.mark.parametrize("scale,noise", [(10, 0.0), (12, 0.1), (14, 0.0), (16, 0.1), (17, 0.0)])
def test_kronecker(scale, noise):
    src, dst = graphgen.kronecker_host(scale, noise=noise, seed=scale)
    _check(src, dst, 1 << scale)


@pytest.mark.parametrize("tau,omega", [(2, 2), (3, 5), (1, 10**7)])
def test_bins(tau, omega):
    src, dst = graphgen.kronecker_host(13, noise=0.1, seed=4)
    _check(src, dst, 1 << 13, tau, omega)


def test_chunglu_and_cliques():
    n = 1 << 15
    prefix, m = graphgen.chunglu_weights(n, 2.1, 30.0)
    s, d = graphgen.chunglu_host(prefix, m, seed=6)
    _check(s, d, n)
    rng = np.random.default_rng(2)
    src, dst = [], []
    for size in np.minimum(3 + rng.zipf(1.7, 3000), 120):
        members = rng.choice(20000, int(size), replace=False)
        for x, y in combinations(members.tolist(), 2):
            src.append(x)
            dst.append(y)
    got = _check(np.asarray(src, np.int32), np.asarray(dst, np.int32), 20000)
    assert got["triangles"] > 10**5


def test_edge_cases():
    # complete graph K_40: C(40, 3) triangles, every wedge closed
    e = np.array(list(combinations(range(40), 2)), np.int32)
    got = _check(e[:, 0].copy(), e[:, 1].copy(), 40)
    assert got["triangles"] == math.comb(40, 3)
    # a star and a path: none
    s = np.zeros(100, np.int32)
    d = np.arange(1, 101, dtype=np.int32)
    assert _check(s, d, 101)["triangles"] == 0
    # no edges at all (only self-loops)
    z = np.arange(10, dtype=np.int32)
    got = _check(z, z, 10)
    assert got["triangles"] == 0 and got["p_total"] == 0


def test_noisy_generator_device_equals_host():
    for scale in (12, 17):
        n_edges = 16 << scale
        s = torch.empty(n_edges, dtype=torch.int32, device="cuda")
        d = torch.empty(n_edges, dtype=torch.int32, device="cuda")
        graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), n_edges, seed=7, noise=0.1)
        torch.cuda.synchronize()
        hs, hd = graphgen.kronecker_host(scale, seed=7, noise=0.1)
        assert np.array_equal(s.cpu().numpy(), hs) and np.array_equal(d.cpu().numpy(), hd)


def test_profile_launches():
    src, dst = graphgen.kronecker_host(14, seed=1)
    g = wedge.graph_build(src, dst, 1 << 14)
    b = wedge.bin(g)
    wedge.profile_enable(False)
    wedge.profile_reset()
    wedge.exact(g, b)
    prof = wedge.profile_read()
    assert prof["exact_orient"]["launches"] == 1 and prof["exact_hash_warp"]["launches"] == 1
    assert prof["scan_degrees"]["launches"] == 1


@pytest.mark.slow
def test_scale24_exact_pins_sampling():
    """Noisy Graph500 scale 24: the sampler's per-bin and global estimates lie
    within Hoeffding's bound (delta = 1e-6 per bin) of the exact values; on the
    plain scale-24 graph, t_i of sampled vertices equals the oracle's
    per-vertex count sum_j |N(i) ∩ N(j)| / 2 from generated rows."""
    scale, n = 24, 1 << 24
    n_edges = 16 << scale
    s = torch.empty(n_edges, dtype=torch.int32, device="cuda")
    d = torch.empty(n_edges, dtype=torch.int32, device="cuda")
    graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), n_edges, seed=3, noise=0.1)
    torch.cuda.synchronize()
    g = wedge.graph_build(s, d, n)
    b = wedge.bin(g, tau=1, omega=2)
    ex = wedge.exact(g, b)
    k = 200_000
    c = wedge.sample(g, b, seed=11, k_per_bin=k, k_global=k)
    eps = math.sqrt(math.log(2 / 1e-6) / (2 * k))
    closed_exact = ex["pbq"][:, 1:].sum(axis=1).astype(np.float64)
    for bi in range(len(ex["p_b"])):
        if ex["p_b"][bi] == 0:
            continue
        c_b = closed_exact[bi] / float(ex["p_b"][bi])
        c_hat = float(c.q[bi, 1:].sum()) / float(c.k_b[bi])
        assert abs(c_hat - c_b) <= eps, (bi, c_hat, c_b)
    c_glob = 3.0 * ex["triangles"] / float(ex["p_total"])
    assert abs(c.closed_global / k - c_glob) <= eps
    del g, b, s, d
    torch.cuda.empty_cache()

    # t_i of sampled vertices on the plain graph, through the oracle's generated rows
    s = torch.empty(n_edges, dtype=torch.int32, device="cuda")
    d = torch.empty(n_edges, dtype=torch.int32, device="cuda")
    graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), n_edges, seed=1)
    torch.cuda.synchronize()
    g = wedge.graph_build(s, d, n)
    b = wedge.bin(g)
    ti = torch.zeros(n, dtype=torch.int64, device="cuda")
    wedge.exact(g, b, t_i=ti)
    deg = torch.zeros(n, dtype=torch.int32, device="cuda")
    g.copy(deg=deg)
    degs = deg.cpu().numpy()
    rng = np.random.default_rng(5)
    cand = np.nonzero((degs >= 2) & (degs <= 300))[0]
    pick = rng.choice(cand, 24, replace=False)
    rows = oracle.rows_kronecker(scale, n_edges, 0.57, 0.19, 0.19, 1, True, pick)
    nbrs = np.unique(np.concatenate([rows[int(v)] for v in pick]))
    rows2 = oracle.rows_kronecker(scale, n_edges, 0.57, 0.19, 0.19, 1, True, nbrs, cap=1 << 27)
    tiv = ti.cpu().numpy()
    for v in pick:
        r = rows[int(v)]
        t = sum(np.intersect1d(r, rows2[int(j)], assume_unique=True).size for j in r) // 2
        assert tiv[v] == t, (int(v), int(tiv[v]), t)
