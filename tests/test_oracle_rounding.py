"""Pins of the oracle's per-vertex allocation by probabilistic rounding (Alg.
Phase 2a) and per-centre draws (Alg. Phase 2c) — CPU only.

q_v must be floor(q*) or ceil(q*) with q* = C(d,2) k_b / p_b (checked in
exact rationals), must equal q* exactly when q* is an integer, and must have
mean q* (the text of Phase 2a: q* = 0.1 gives one sample with probability
0.1 — the opposite rule fails here). The tallies must estimate the exact
per-bin clustering coefficients (Thm 3.2) within Hoeffding's bound.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import graphgen
import oracle


def _graph(edges, n):
    e = np.asarray(edges, np.int32).reshape(-1, 2)
    return oracle.csr(e[:, 0], e[:, 1], n)


def test_q_is_floor_or_ceil_of_ideal_share():
    src, dst = graphgen.kronecker_host(10, seed=4)
    off, adj = oracle.csr(src, dst, 1 << 10)
    deg = oracle.degrees(off).astype(np.int64)
    for tau, omega, k in [(1, 2, 1000), (2, 2, 77), (3, 5, 123456)]:
        r = oracle.sample_rounding(off, adj, tau, omega, seed=9, k_per_bin=k, per_vertex=True)
        p_b = {}
        for d in deg:
            if d >= 2:
                b = oracle.bin_id(int(d), tau, omega)
                p_b[b] = p_b.get(b, 0) + int(d) * (int(d) - 1) // 2
        for v, d in enumerate(deg):
            q = int(r["qv"][v])
            if d < 2:
                assert q == 0
                continue
            qs = Fraction(int(d) * (int(d) - 1) // 2 * k, p_b[oracle.bin_id(int(d), tau, omega)])
            assert q in (math.floor(qs), math.ceil(qs))
        # realised totals are the sums of q_v per bin
        for b, row in enumerate(r["counts"]):
            members = [v for v, d in enumerate(deg) if d >= 2 and oracle.bin_id(int(d), tau, omega) == b]
            assert int(row[0]) == int(sum(int(r["qv"][v]) for v in members))
            assert int(row[0]) == int(row[1:].sum())


def test_integer_share_is_exact():
    """Cycle C_12: every vertex has d = 2, one wedge, p_b = 12; k = 36 gives q* = 3 for every vertex.
    No triangles, so all 36 samples are open. Triangle K_3: every sample closed, class 3."""
    off, adj = _graph([(i, (i + 1) % 12) for i in range(12)], 12)
    r = oracle.sample_rounding(off, adj, 1, 2, seed=1, k_per_bin=36, per_vertex=True)
    assert list(r["qv"]) == [3] * 12
    assert list(r["counts"][2]) == [36, 36, 0, 0, 0]
    off, adj = _graph([(0, 1), (1, 2), (0, 2)], 3)
    r = oracle.sample_rounding(off, adj, 1, 2, seed=2, k_per_bin=30, per_vertex=True)
    assert list(r["qv"]) == [10, 10, 10]
    assert list(r["counts"][2]) == [30, 0, 0, 0, 30]


def test_rounding_probability_is_the_fraction():
    """Path a-b-c (b has d = 2, one wedge) and a star with centre d = 3 (three wedges) share
    bin 2 (2 <= d < 4) with p_b = 4. With k = 1: q*(b) = 1/4, q*(centre) = 3/4."""
    off, adj = _graph([(0, 1), (1, 2), (3, 4), (3, 5), (3, 6)], 7)
    seeds = 2000
    qb = np.zeros(seeds)
    qc = np.zeros(seeds)
    for s in range(seeds):
        r = oracle.sample_rounding(off, adj, 1, 2, seed=1000 + s, k_per_bin=1, per_vertex=True)
        qb[s], qc[s] = r["qv"][1], r["qv"][3]
    eps = math.sqrt(math.log(2 / 1e-9) / (2 * seeds))  # Hoeffding, delta = 1e-9
    assert abs(qb.mean() - 0.25) <= eps and abs(qc.mean() - 0.75) <= eps
    assert set(np.unique(qb)) <= {0, 1} and set(np.unique(qc)) <= {0, 1}


def test_estimates_match_exact_clustering():
    """Thm 3.2 with the realised k_b: |c_hat_b - c_b| within Hoeffding's bound in every bin."""
    src, dst = graphgen.kronecker_host(11, seed=6)
    off, adj = oracle.csr(src, dst, 1 << 11)
    ex = oracle.exact(off, adj, 1, 2)
    k = 40000
    r = oracle.sample_rounding(off, adj, 1, 2, seed=5, k_per_bin=k)
    p_b = ex["p_b"]
    for b, row in enumerate(r["counts"]):
        kb = int(row[0])
        if p_b[b] == 0:
            assert kb == 0
            continue
        c_exact = sum(int(x) for x in ex["pbq"][b][1:]) / int(p_b[b])
        c_hat = (int(row[2]) + int(row[3]) + int(row[4])) / kb
        eps = math.sqrt(math.log(2 / 1e-7) / (2 * kb))
        assert abs(c_hat - c_exact) <= eps, (b, c_hat, c_exact)
        # the per-class counts estimate p_{b,q} / p_b too
        for q in (1, 2, 3):
            assert abs(int(row[1 + q]) / kb - int(ex["pbq"][b][q]) / int(p_b[b])) <= eps


def test_budget_per_bin_and_zero_budget():
    src, dst = graphgen.kronecker_host(9, seed=7)
    off, adj = oracle.csr(src, dst, 1 << 9)
    nb = oracle.n_bins_for(off, 1, 2)
    kb = np.zeros(nb, np.uint64)
    kb[3] = 5000
    r = oracle.sample_rounding(off, adj, 1, 2, seed=3, k_per_bin=0, k_bins=kb, per_vertex=True)
    rows = r["counts"]
    assert all(int(rows[b][0]) == 0 for b in range(nb) if b != 3)
    assert abs(int(rows[3][0]) - 5000) <= math.sqrt(nb * 1e3)  # a sum of independent 0/1 roundings
