"""Pins of the CPU oracle to facts the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/), closed forms, invariants, an independent
library (networkx) or brute force on tiny graphs.
"""
import json
import math
import os
from itertools import combinations

import numpy as np
import pytest

import graphgen
import oracle
from oracle import brute
from oracle.estimate import estimate

from conftest import GOLDEN

nx = pytest.importorskip("networkx")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _graph_from_nx(G, n):
    src = np.array([u for u, v in G.edges()], np.int32)
    dst = np.array([v for u, v in G.edges()], np.int32)
    return oracle.csr(src, dst, n)


# ---------------------------------------------------------------------------
# Worked example of Sec. 2.2 (Fig. example)
# ---------------------------------------------------------------------------

def test_fig_example_degrees_wedges_triangles():
    g = _load("fig_example.json")
    e = np.array(g["edges"], np.int32)
    off, adj = oracle.csr(e[:, 0], e[:, 1], g["n"])
    d = np.diff(off)
    assert d.tolist() == g["d"]
    assert adj.shape[0] == 2 * g["m"]
    assert [x * (x - 1) // 2 for x in d.tolist()] == g["p_i"]
    ex = oracle.exact(off, adj, tau=10, omega=2)  # tau >= 4: singleton bins
    assert ex["t"] == g["t"]
    assert ex["t_i"].tolist() == g["t_i"]
    p = int(sum(g["p_i"]))
    assert p == g["p"]
    assert 3 * ex["t"] / p == pytest.approx(g["c"], abs=0)
    c_i = [ti / pi if pi else 0 for ti, pi in zip(ex["t_i"].tolist(), g["p_i"])]
    assert c_i == pytest.approx(g["c_i"], abs=1e-15)


def test_fig_example_singleton_bins():
    g = _load("fig_example.json")
    e = np.array(g["edges"], np.int32)
    off, adj = oracle.csr(e[:, 0], e[:, 1], g["n"])
    ex = oracle.exact(off, adj, tau=10, omega=2)
    for i, D in enumerate(g["singleton_bins"]):
        assert oracle.bin_id(D, 10, 2) == D
        assert int(ex["n_b"][D]) == g["n_d"][i]
        assert int(ex["p_b"][D]) == g["p_d"][i]
        pbq = [int(x) for x in ex["pbq"][D]]
        t_d = pbq[1] + pbq[2] / 2 + pbq[3] / 3
        assert t_d == pytest.approx(g["t_d"][i], abs=1e-15)
        c_d = (pbq[1] + pbq[2] + pbq[3]) / g["p_d"][i] if g["p_d"][i] else 0.0
        assert c_d == pytest.approx(g["c_d"][i], abs=1e-15)


def test_fig_example_estimators_on_exhaustive_sample():
    """Feeding every wedge once (k_b = p_b) into the estimators of Thm 3.2 and
    Thm 3.3 must reproduce the printed c_d and t_d exactly."""
    g = _load("fig_example.json")
    e = np.array(g["edges"], np.int32)
    off, adj = oracle.csr(e[:, 0], e[:, 1], g["n"])
    tau, omega = 10, 2
    nb = oracle.n_bins_for(off, tau, omega)
    d = np.diff(off)
    v0, v1, v2 = [], [], []
    for c in range(g["n"]):
        for i, j in combinations(adj[off[c]:off[c + 1]].tolist(), 2):
            v0.append(c), v1.append(i), v2.append(j)
    q = oracle.classify(off, adj, tau, omega, v0, v1, v2)
    counts = np.zeros((nb, 5), np.uint64)
    for c, qq in zip(v0, q.tolist()):
        b = oracle.bin_id(int(d[c]), tau, omega)
        counts[b, 0] += 1
        counts[b, 1 + qq] += 1
    bb = oracle.bins(off, tau, omega)
    est = estimate(bb["p_b"], counts, [0, 0], delta=0.1)
    for i, D in enumerate(g["singleton_bins"]):
        assert est["c_b"][D] == pytest.approx(g["c_d"][i], abs=1e-15)
        assert est["t_b"][D] == pytest.approx(g["t_d"][i], abs=1e-12)
    assert est["c_hat"] == pytest.approx(g["c"], abs=1e-15)  # Eq. (global_est) with exact c_b
    assert est["t_hat"] == pytest.approx(g["t"], abs=1e-12)


# ---------------------------------------------------------------------------
# Binning (Sec. 4.2)
# ---------------------------------------------------------------------------

def test_printed_bins_tau2_omega2():
    g = _load("bins_printed.json")
    for k, (lo, hi) in enumerate(g["tau2_omega2"], start=1):
        assert oracle.bin_lodeg(k, 2, 2) == lo
        assert oracle.bin_lodeg(k + 1, 2, 2) - 1 == hi
        for d in range(lo, hi + 1):
            assert oracle.bin_id(d, 2, 2) == k


@pytest.mark.parametrize("dbar", [7, 100, 10**7])
def test_single_bin_and_singletons(dbar):
    # tau=1, omega=dbar: {1}, {2..dbar}
    assert oracle.bin_lodeg(2, 1, dbar) == 2
    assert oracle.bin_lodeg(3, 1, dbar) - 1 >= dbar
    for d in [2, 3, dbar // 2 + 1, dbar]:
        assert oracle.bin_id(d, 1, dbar) == 2
    # tau=dbar: every bin a singleton
    for d in [1, 2, 3, min(dbar, 1000)]:
        assert oracle.bin_id(d, dbar, 2) == d


def test_tau1_omega2_is_power_of_two_bins():
    """tau=1, omega=2 gives bins 2^i <= d < 2^(i+1), bin id i+1."""
    for d in list(range(1, 5000)) + [2**20 - 1, 2**20, 2**30, 2**31 - 1]:
        assert oracle.bin_id(d, 1, 2) == d.bit_length()


@pytest.mark.parametrize("tau,omega", [(1, 2), (2, 2), (3, 3), (1, 10), (5, 7), (2, 1000)])
def test_binid_binlodeg_consistent(tau, omega):
    k = 1
    while True:
        lo, lo_next = oracle.bin_lodeg(k, tau, omega), oracle.bin_lodeg(k + 1, tau, omega)
        if lo_next > 2**31:
            break
        assert lo < lo_next
        assert oracle.bin_id(lo, tau, omega) == k
        assert oracle.bin_id(lo_next - 1, tau, omega) == k
        k += 1


@pytest.mark.parametrize("tau,omega", [(1, 2), (2, 2), (3, 3), (1, 10), (4, 5)])
def test_binid_matches_paper_log_formula(tau, omega):
    """Eq. (BinId) in floating point agrees with the exact integer form away
    from exact powers of omega, where a float log may round either way."""
    for d in range(1, 20000):
        if d <= tau:
            assert oracle.bin_id(d, tau, omega) == d
            continue
        x = 1 + (omega - 1) * (d - tau)
        m = int(math.floor(math.log(x) / math.log(omega)))
        exact_power = any(omega**j == x or omega**j == x + 1 for j in range(0, 64))
        if not exact_power:
            assert oracle.bin_id(d, tau, omega) == m + tau


# ---------------------------------------------------------------------------
# Random words and sample budget
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    g = _load("philox_kat.json")
    for v in g["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_hoeffding_budget():
    # Sec. 5.3: at 99.9% confidence, k = 2000 samples give error eps = 0.05.
    assert oracle.hoeffding_k(0.05, 0.001) <= 2000
    for eps, delta in [(0.002, 0.001), (0.01, 0.001), (0.005, 0.001), (0.05, 0.1), (0.3, 0.5)]:
        k = oracle.hoeffding_k(eps, delta)
        bound = math.log(2 / delta) / (2 * eps * eps)
        assert k >= bound and k - 1 < bound  # the smallest integer k satisfying Thm 3.1
    assert oracle.hoeffding_k(0.002, 0.001) == 950113  # ln(2000)/(8e-6) = 950112.81 -> 950113
    assert oracle.hoeffding_k(0.0, 0.1) == 0  # invalid eps


# ---------------------------------------------------------------------------
# CSR and exact counts against networkx and brute force
# ---------------------------------------------------------------------------

def _random_multigraph(rng, n, m):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    # duplicates, reversed duplicates and self-loops on purpose
    src = np.concatenate([src, dst[: m // 4], src[: m // 8], np.arange(3, dtype=np.int32)])
    dst = np.concatenate([dst, src[: m // 4], dst[: m // 8], np.arange(3, dtype=np.int32)])
    return src, dst


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_csr_matches_networkx(seed):
    rng = np.random.default_rng(seed)
    n, m = 300, 2000
    src, dst = _random_multigraph(rng, n, m)
    off, adj = oracle.csr(src, dst, n)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((int(u), int(v)) for u, v in zip(src, dst) if u != v)
    for v in range(n):
        assert adj[off[v]:off[v + 1]].tolist() == sorted(G.neighbors(v))


def test_csr_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.csr([0, 5], [1, 2], 5)
    with pytest.raises(ValueError):
        oracle.csr([0, -1], [1, 2], 5)


def test_csr_empty_graph():
    off, adj = oracle.csr(np.zeros(0, np.int32), np.zeros(0, np.int32), 4)
    assert off.tolist() == [0, 0, 0, 0, 0] and adj.shape[0] == 0


@pytest.mark.parametrize("seed", [3, 4])
def test_exact_matches_networkx(seed):
    rng = np.random.default_rng(seed)
    n, m = 400, 4000
    src, dst = _random_multigraph(rng, n, m)
    off, adj = oracle.csr(src, dst, n)
    ex = oracle.exact(off, adj, 2, 2)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((int(u), int(v)) for u, v in zip(src, dst) if u != v)
    tri = nx.triangles(G)
    assert ex["t_i"].tolist() == [tri[v] for v in range(n)]
    assert ex["t"] * 3 == sum(tri.values())  # sum_i t_i = 3t (Sec. 2.1)
    p = int(ex["p_b"].sum())
    assert 3 * ex["t"] / p == pytest.approx(nx.transitivity(G), rel=1e-12)  # Eq. (CC)


@pytest.mark.parametrize("seed,tau,omega", [(5, 2, 2), (6, 1, 2), (7, 3, 3), (8, 30, 2)])
def test_exact_pbq_matches_brute_force(seed, tau, omega):
    rng = np.random.default_rng(seed)
    n = 24
    src, dst = _random_multigraph(rng, n, 90)
    off, adj = oracle.csr(src, dst, n)
    ex = oracle.exact(off, adj, tau, omega)
    bf = brute.counts(brute.edge_set(src, dst), n, lambda d: oracle.bin_id(d, tau, omega))
    assert ex["t"] == bf["t"]
    assert ex["t_i"].tolist() == bf["t_i"]
    for D, row in bf["pdq"].items():
        assert [int(x) for x in ex["pbq"][D]] == row
    # every closed wedge lands in exactly one (bin, q >= 1) cell: sum = 3t
    assert int(ex["pbq"][:, 1:].sum()) == 3 * ex["t"]


def test_single_bin_triangles_equal_total():
    """One bin of all degrees (tau=1, omega=dbar): every closed wedge has all
    three vertices in the bin, so t_D = p_{D,3}/3 = t."""
    src, dst = graphgen.kronecker_host(9)
    off, adj = oracle.csr(src, dst, 512)
    ex = oracle.exact(off, adj, 1, 10**7)
    assert int(ex["pbq"][2, 1]) == 0 and int(ex["pbq"][2, 2]) == 0
    assert int(ex["pbq"][2, 3]) == 3 * ex["t"]


@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_complete_graph(n):
    G = nx.complete_graph(n)
    off, adj = _graph_from_nx(G, n)
    ex = oracle.exact(off, adj, 2, 2)
    assert ex["t"] == math.comb(n, 3)
    assert 3 * ex["t"] / int(ex["p_b"].sum()) == 1.0


@pytest.mark.parametrize("G,n", [(nx.star_graph(9), 10), (nx.complete_bipartite_graph(4, 6), 10),
                                 (nx.cycle_graph(8), 8), (nx.path_graph(9), 9)])
def test_triangle_free_graphs(G, n):
    off, adj = _graph_from_nx(G, n)
    ex = oracle.exact(off, adj, 2, 2)
    assert ex["t"] == 0
    r = oracle.sample(off, adj, 2, 2, seed=3, k_per_bin=500, k_global=500)
    assert int(r["counts"][:, 2:].sum()) == 0 and int(r["glob"][1]) == 0


def test_triangle_cycle():
    off, adj = _graph_from_nx(nx.cycle_graph(3), 3)
    ex = oracle.exact(off, adj, 2, 2)
    assert ex["t"] == 1
    r = oracle.sample(off, adj, 2, 2, seed=3, k_per_bin=100, k_global=100)
    assert int(r["glob"][1]) == 100  # every wedge of a triangle is closed


# ---------------------------------------------------------------------------
# Sampling (Sec. 3.2, Thm 3.2, Thm 3.3)
# ---------------------------------------------------------------------------

def test_exhaustive_classification_equals_exact():
    """Classifying every wedge once reproduces the exact p_{b,q}."""
    src, dst = graphgen.kronecker_host(8)
    off, adj = oracle.csr(src, dst, 256)
    tau, omega = 2, 2
    ex = oracle.exact(off, adj, tau, omega)
    d = np.diff(off)
    v0, v1, v2 = [], [], []
    for c in range(256):
        row = adj[off[c]:off[c + 1]].tolist()
        for i, j in combinations(row, 2):
            v0.append(c), v1.append(i), v2.append(j)
    q = oracle.classify(off, adj, tau, omega, v0, v1, v2)
    nb = oracle.n_bins_for(off, tau, omega)
    pbq = np.zeros((nb, 4), np.uint64)
    for c, qq in zip(v0, q.tolist()):
        pbq[oracle.bin_id(int(d[c]), tau, omega), qq] += 1
    assert (pbq == ex["pbq"]).all()


@pytest.mark.parametrize("tau,omega", [(1, 2), (2, 2)])
def test_estimates_within_hoeffding_bound(tau, omega):
    """Thm 3.2 and Thm 3.3 with k = Hoeffding(eps, delta): |c_hat_b - c_b| < eps
    and |t_hat_b - t_b| < eps p_b for every bin (fixed seed: deterministic)."""
    src, dst = graphgen.kronecker_host(12)
    off, adj = oracle.csr(src, dst, 4096)
    eps, delta = 0.01, 0.001
    k = oracle.hoeffding_k(eps, delta)
    r = oracle.sample(off, adj, tau, omega, seed=7, k_per_bin=k, k_global=k)
    ex = oracle.exact(off, adj, tau, omega)
    est = estimate(ex["p_b"], r["counts"], r["glob"], delta)
    for b in range(ex["pbq"].shape[0]):
        pb = int(ex["p_b"][b])
        if pb == 0:
            assert int(r["counts"][b, 0]) == 0
            continue
        assert int(r["counts"][b, 0]) == k and int(r["counts"][b, 1:].sum()) == k
        pbq = [int(x) for x in ex["pbq"][b]]
        c_b = (pbq[1] + pbq[2] + pbq[3]) / pb
        t_b = pbq[1] + pbq[2] / 2 + pbq[3] / 3
        assert abs(est["c_b"][b] - c_b) < eps
        assert abs(est["t_b"][b] - t_b) < eps * pb
    c = 3 * ex["t"] / int(ex["p_b"].sum())
    assert abs(est["c_hat_global"] - c) < eps
    assert abs(est["c_hat"] - c) < eps


def _cliques_with_pendants(n_cliques, seed):
    """n_cliques copies of K_8 in which four "heavy" members each carry five
    pendant leaves (degree 12, bin 4 with tau = 1, omega = 2) and the other
    four are plain (degree 7, bin 3); vertex ids shuffled."""
    rng = np.random.default_rng(seed)
    n = n_cliques * (8 + 4 * 5)
    perm = rng.permutation(n).astype(np.int32)
    src, dst = [], []
    leaf = n_cliques * 8
    for c in range(n_cliques):
        members = [8 * c + i for i in range(8)]
        for a, b in combinations(members, 2):
            src.append(a)
            dst.append(b)
        for h in members[:4]:
            for _ in range(5):
                src.append(h)
                dst.append(leaf)
                leaf += 1
    return perm[np.array(src)], perm[np.array(dst)], n


def test_class_fractions_per_bin_match_closed_form():
    """Thm 3.3 / Alg. Phase 4c classes, per bin, by closed form. A plain
    centre (bin 3) has 21 wedges: both ends plain (3, class 3), one heavy (12,
    class 2), both heavy (6, class 1), all closed. A heavy centre (bin 4) has
    66: heavy-heavy 3 (class 3), heavy-plain 12 (class 2), plain-plain 6
    (class 1), and 45 with a leaf, open (class 0). The exact enumeration and
    the sampler's class fractions q_c / k_b must both agree; classes 2 and 3
    differ by far more than the Hoeffding radius, so exchanging them (or any
    two classes) fails."""
    src, dst, n = _cliques_with_pendants(60, seed=11)
    off, adj = oracle.csr(src, dst, n)
    want = {3: np.array([0, 6, 12, 3]) / 21.0, 4: np.array([45, 6, 12, 3]) / 66.0}
    ex = oracle.exact(off, adj, 1, 2)
    centres = {3: 4 * 60, 4: 4 * 60}
    for b, frac in want.items():
        assert int(ex["p_b"][b]) == centres[b] * (21 if b == 3 else 66)
        assert np.array_equal(ex["pbq"][b].astype(np.int64), np.rint(frac * int(ex["p_b"][b])).astype(np.int64))
    k = 40000
    r = oracle.sample(off, adj, 1, 2, seed=13, k_per_bin=k, k_global=0)
    eps = math.sqrt(math.log(2 / 1e-7) / (2 * k))
    for b, frac in want.items():
        row = r["counts"][b]
        assert int(row[0]) == k
        got = np.array([int(x) for x in row[1:]]) / k
        assert np.all(np.abs(got - frac) <= eps), (b, got, frac)
        # the test's power: exchanging classes 2 and 3 moves both fractions by > 2 eps
        assert abs(frac[2] - frac[3]) > 2 * eps
    # bins without wedges get no samples
    assert all(int(r["counts"][b][0]) == 0 for b in range(len(r["counts"])) if b not in want)


def test_centre_distribution_chi_square():
    """Centres of the global stream are drawn with probability C(d,2)/p (Sec. 3.2)."""
    from scipy.stats import chisquare
    src, dst = graphgen.kronecker_host(6)
    off, adj = oracle.csr(src, dst, 64)
    k = 200000
    r = oracle.sample(off, adj, 2, 2, seed=11, k_per_bin=0, k_global=k, records=True)
    d = np.diff(off)
    w = d * (d - 1) // 2
    obs = np.bincount(r["records"][:, 0], minlength=64)
    mask = w > 0
    assert (obs[~mask] == 0).all()
    exp = w[mask] / w.sum() * k
    assert chisquare(obs[mask], exp).pvalue > 1e-4


def test_neighbour_pair_distribution_chi_square():
    """For a fixed centre, the unordered endpoint pair is uniform over its C(d,2) pairs."""
    from scipy.stats import chisquare
    G = nx.star_graph(12)  # centre 0 with 12 leaves: the only wedge centre
    off, adj = _graph_from_nx(G, 13)
    k = 66 * 2000
    r = oracle.sample(off, adj, 2, 2, seed=5, k_per_bin=0, k_global=k, records=True)
    rec = r["records"]
    assert (rec[:, 0] == 0).all() and (rec[:, 1] != rec[:, 2]).all()
    pairs = np.minimum(rec[:, 1], rec[:, 2]) * 13 + np.maximum(rec[:, 1], rec[:, 2])
    _, obs = np.unique(pairs, return_counts=True)
    assert obs.shape[0] == 66
    assert chisquare(obs).pvalue > 1e-4


def test_records_are_valid_wedges():
    src, dst = graphgen.kronecker_host(10)
    off, adj = oracle.csr(src, dst, 1024)
    r = oracle.sample(off, adj, 1, 2, seed=9, k_per_bin=100, k_global=5000, records=True)
    rec = r["records"]
    nbs = [set(adj[off[v]:off[v + 1]].tolist()) for v in range(1024)]
    for v0, v1, v2, closed, d0, d1, d2, _ in rec.tolist():
        assert v1 in nbs[v0] and v2 in nbs[v0] and v1 != v2
        assert closed == (v2 in nbs[v1])
        assert (d0, d1, d2) == (len(nbs[v0]), len(nbs[v1]), len(nbs[v2]))
    assert int(r["stats"].sum()) == int(r["glob"][1]) == int(rec[:, 3].sum())


def test_seeds_change_samples_and_repeat_exactly():
    src, dst = graphgen.kronecker_host(10)
    off, adj = oracle.csr(src, dst, 1024)
    a = oracle.sample(off, adj, 1, 2, seed=1, k_per_bin=1000, k_global=1000)
    b = oracle.sample(off, adj, 1, 2, seed=1, k_per_bin=1000, k_global=1000)
    c = oracle.sample(off, adj, 1, 2, seed=2, k_per_bin=1000, k_global=1000)
    assert (a["counts"] == b["counts"]).all() and (a["glob"] == b["glob"]).all()
    assert not (a["counts"] == c["counts"]).all()


# ---------------------------------------------------------------------------
# Input generator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 1000, 1024, 4097])
def test_feistel_is_a_bijection(n):
    y = graphgen.permute_host(n, 12345, np.arange(n, dtype=np.uint64))
    assert sorted(y.tolist()) == list(range(n))


def test_rmat_quadrant_frequencies():
    """Without permutation, the top bits follow the generator matrix: P(u's
    top bit = 1) = c + d = 0.24 and P(v's top bit = 1) = b + d = 0.24."""
    S = 16
    src, dst = graphgen.kronecker_host(S, n_edges=400000, permute=False)
    fu = float(((src >> (S - 1)) & 1).mean())
    fv = float(((dst >> (S - 1)) & 1).mean())
    both = float((((src >> (S - 1)) & 1) & ((dst >> (S - 1)) & 1)).mean())
    assert abs(fu - 0.24) < 0.005 and abs(fv - 0.24) < 0.005 and abs(both - 0.05) < 0.003


def test_generator_ranges_and_chunking():
    src, dst = graphgen.kronecker_host(12)
    assert src.shape[0] == 16 * 4096
    assert src.min() >= 0 and src.max() < 4096 and dst.min() >= 0 and dst.max() < 4096
    s2, d2 = graphgen.kronecker_host(12, n_edges=1000, e0=5000)
    assert (s2 == src[5000:6000]).all() and (d2 == dst[5000:6000]).all()


def test_rows_from_generator_match_csr():
    S = 11
    src, dst = graphgen.kronecker_host(S)
    off, adj = oracle.csr(src, dst, 1 << S)
    q = [0, 5, 77, 1000, 2047]
    rows = oracle.rows_kronecker(S, 16 << S, 0.57, 0.19, 0.19, 1, True, q)
    for v in q:
        assert rows[v].tolist() == adj[off[v]:off[v + 1]].tolist()


def test_chunglu_generator():
    prefix, m = graphgen.chunglu_weights(1024, 2.3, 16.0)
    assert m == 1024 * 8
    assert (np.diff(prefix.astype(np.int64)) > 0).all()
    src, dst = graphgen.chunglu_host(prefix, m, seed=3)
    assert src.min() >= 0 and src.max() < 1024
    off, adj = oracle.csr(src, dst, 1024)
    assert adj.shape[0] > 0
