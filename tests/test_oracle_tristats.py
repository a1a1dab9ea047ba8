"""Pins of the oracle's triangle statistics (Sec. 5.7, Thm 3.4) — CPU only.

The box-plot rule is checked against hand-worked cases and numpy's
inverted-CDF percentiles; the sampled statistics against graphs whose
triangles are known in closed form (complete, bipartite, windmill) and, on
a random graph, against brute-force triangle enumeration: every triangle has
three closed wedges with the same (d_min, d_max), so the fraction of samples
that are closed with d_min in bin a and d_max in bin b is 3 T_ab / p.
"""
import json
import os
import math
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import graphgen
import oracle
from oracle import tristats

from conftest import GOLDEN


def _graph(edges, n):
    e = np.asarray(edges, np.int32).reshape(-1, 2)
    return oracle.csr(e[:, 0], e[:, 1], n)


def test_box_golden_cases():
    g = json.load(open(os.path.join(GOLDEN, "boxplot_cases.json")))
    assert g["fields"] == list(tristats.BOX_FIELDS)
    for case in g["cases"]:
        s = tristats.box(case["values"])
        assert [s[f] for f in g["fields"]] == case["expect"], case["why"]


def test_nearest_rank_matches_numpy_inverted_cdf():
    rng = np.random.default_rng(11)
    for _ in range(500):
        c = int(rng.integers(1, 60))
        v = np.sort(rng.integers(0, 1000, c))
        for p in (Fraction(1, 4), Fraction(1, 2), Fraction(3, 4)):
            assert tristats.nearest_rank(list(v), p) == np.percentile(v, float(p) * 100, method="inverted_cdf")


def test_whiskers_by_float_bounds():
    """Whiskers and outliers against bounds computed in FP64 (exact here: small integers and halves)."""
    rng = np.random.default_rng(12)
    for _ in range(300):
        c = int(rng.integers(1, 40))
        v = rng.integers(2, 200, c)
        if rng.random() < 0.3:
            v[: c // 3] = rng.integers(1000, 5000, c // 3)  # a heavy tail
        s = tristats.box(v)
        q1 = np.percentile(v, 25, method="inverted_cdf")
        q3 = np.percentile(v, 75, method="inverted_cdf")
        lo, hi = q1 - 1.5 * (q3 - q1), q3 + 1.5 * (q3 - q1)
        inside = v[(v >= lo) & (v <= hi)]
        assert s["whisker_lo"] == inside.min() and s["whisker_hi"] == inside.max()
        assert s["outliers"] == c - inside.size
        assert s["min"] == v.min() and s["max"] == v.max() and s["count"] == c


def test_complete_graph_every_sample_is_a_triangle():
    n = 6
    off, adj = _graph(list(combinations(range(n), 2)), n)
    k = 5000
    r = tristats.triangle_stats(off, adj, seed=3, k=k)
    assert r["closed"] == k
    # degree 5: BinLoDeg(4) = 2^2 + 1 = 5 <= 5 < BinLoDeg(5) = 9 (tau = 2, omega = 2)
    expect = np.zeros((oracle.STAT_BINS, 9), np.uint64)
    expect[4] = [k, 5, 5, 5, 5, 5, 5, 5, 0]
    assert np.array_equal(r["box"], expect)
    assert list(r["ratio_q"]) == [1.0] * 5
    assert r["hist"][4, 4] == k and r["hist"].sum() == k
    assert np.array_equal(r["hist"], r["stats"])


def test_bipartite_graph_has_no_triangles():
    off, adj = _graph([(a, 3 + b) for a in range(3) for b in range(4)], 7)
    r = tristats.triangle_stats(off, adj, seed=4, k=3000)
    assert r["closed"] == 0 and not r["box"].any() and not r["ratio_q"].any() and not r["hist"].any()


@pytest.mark.parametrize("blades", [3, 10])
def test_windmill(blades):
    """Windmill: `blades` triangles sharing a centre of degree 2 blades; leaves have degree 2.
    Every triangle has d_min = 2 (bin 2), d_max = 2 blades, ratio blades. Wedges:
    2 blades at the leaves (all closed) + C(2 blades, 2) at the centre (blades closed),
    so c = 3 blades / (2 blades + blades (2 blades - 1)) = 3 / (2 blades + 1)."""
    n = 2 * blades + 1
    edges = []
    for i in range(blades):
        a, b = 1 + 2 * i, 2 + 2 * i
        edges += [(0, a), (0, b), (a, b)]
    off, adj = _graph(edges, n)
    k = 40000
    r = tristats.triangle_stats(off, adj, seed=5, k=k)
    c = r["closed"]
    eps = math.sqrt(math.log(2 / 1e-9) / (2 * k))  # Thm 3.1 at delta = 1e-9
    assert abs(c / k - 3 / (2 * blades + 1)) <= eps
    d = 2 * blades
    expect = np.zeros((oracle.STAT_BINS, 9), np.uint64)
    expect[2] = [c, d, d, d, d, d, d, d, 0]
    assert np.array_equal(r["box"], expect)
    assert list(r["ratio_q"]) == [float(blades)] * 5


def _triangles(off, adj):
    n = off.shape[0] - 1
    nb = [set(adj[off[i]:off[i + 1]].tolist()) for i in range(n)]
    out = []
    for a in range(n):
        hi = sorted(x for x in nb[a] if x > a)
        for b, c in combinations(hi, 2):
            if c in nb[b]:
                out.append((a, b, c))
    return out


def test_closed_samples_are_uniform_triangles():
    """Thm 3.4 through the (BinId(d_min), BinId(d_max)) histogram, every cell within Hoeffding's bound."""
    src, dst = graphgen.kronecker_host(9, seed=21)
    off, adj = oracle.csr(src, dst, 1 << 9)
    deg = oracle.degrees(off)
    p = int(sum(int(d) * (int(d) - 1) // 2 for d in deg))
    cells = np.zeros((oracle.STAT_BINS, oracle.STAT_BINS), np.int64)
    for t in _triangles(off, adj):
        ds = sorted(int(deg[v]) for v in t)
        cells[oracle.bin_id(ds[0], 2, 2), oracle.bin_id(ds[2], 2, 2)] += 1
    assert cells.sum() > 100
    k = 2_000_000
    s = oracle.sample(off, adj, 1, 2, 77, 0, k)
    hist = s["stats"].astype(np.int64)
    eps = math.sqrt(math.log(2 * cells.size / 1e-6) / (2 * k))
    assert np.all(np.abs(hist / k - 3 * cells / p) <= eps)
    assert int(s["glob"][1]) == hist.sum()
    # and with the same samples' records, summarise() rebuilds that histogram
    r = tristats.triangle_stats(off, adj, seed=77, k=200_000)
    assert np.array_equal(r["hist"], r["stats"]) and r["closed"] == int(r["hist"].sum())
    # every group's box ends at the group's extremes, over the triangles' own values
    for b in range(oracle.STAT_BINS):
        cnt = r["box"][b, 0]
        assert cnt == r["hist"][b].sum()
        if cnt:
            assert r["box"][b, 1] <= r["box"][b, 2] <= r["box"][b, 3] <= r["box"][b, 4] <= r["box"][b, 5]
