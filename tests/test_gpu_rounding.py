"""WEDGE_FLAG_ROUNDING (Alg. Phase 2a allocation, Alg. Phase 2c draws) on
GB300 against the oracle: realised per-bin totals and q0..q3 tallies must be
identical; the global stream must be unchanged by the flag.
"""
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


def _compare(src, dst, n, tau, omega, seed, k, k_bin=None, k_global=0):
    g = wedge.graph_build(src, dst, n)
    b = wedge.bin(g, tau=tau, omega=omega)
    flags = wedge.FLAG_ROUNDING | (0 if k_global else wedge.FLAG_NO_GLOBAL)
    got = wedge.sample(g, b, seed=seed, k_per_bin=k, k_global=k_global, flags=flags, k_bin=k_bin)
    off, adj = oracle.csr(src, dst, n)
    ref = oracle.sample_rounding(off, adj, tau, omega, seed, k, k_bins=k_bin)
    assert np.array_equal(got.counts_matrix(), ref["counts"])
    if k_global:
        plain = oracle.sample(off, adj, tau, omega, seed, 0, k_global)
        assert got.k_global == k_global and got.closed_global == int(plain["glob"][1])
        assert np.array_equal(got.stats, plain["stats"])
    return got


@pytest.mark.parametrize("scale,tau,omega,k", [(10, 1, 2, 5000), (12, 1, 2, 100_000), (12, 2, 2, 20_000),
                                               (11, 3, 5, 7777), (13, 1, 2, 3)])
def test_kronecker(scale, tau, omega, k):
    src, dst = graphgen.kronecker_host(scale, seed=scale + tau)
    _compare(src, dst, 1 << scale, tau, omega, 40 + scale, k, k_global=1000)


def test_chunglu_heavy_tail():
    n = 1 << 14
    prefix, m = graphgen.chunglu_weights(n, 2.0, 20.0)
    s, d = graphgen.chunglu_host(prefix, m, seed=3)
    _compare(s, d, n, 1, 2, 11, 250_000)


def test_per_bin_budgets_and_zeros():
    src, dst = graphgen.kronecker_host(12, seed=5)
    g = wedge.graph_build(src, dst, 1 << 12)
    nb = wedge.bin(g).info().n_bins
    kb = np.zeros(nb, np.uint64)
    kb[2::2] = 3000
    kb[nb - 1] = 1 << 20  # the top bin: a few vertices with huge shares
    _compare(src, dst, 1 << 12, 1, 2, 8, 0, k_bin=kb)


def test_integer_shares_and_no_triangles():
    e = np.array([(i, (i + 1) % 1000) for i in range(1000)], np.int32)  # cycle: q* = k / 1000
    got = _compare(e[:, 0].copy(), e[:, 1].copy(), 1000, 1, 2, 1, 7000)
    assert list(got.counts_matrix()[2]) == [7000, 7000, 0, 0, 0]


def test_flag_errors():
    src, dst = graphgen.kronecker_host(9, seed=1)
    g = wedge.graph_build(src, dst, 1 << 9)
    b = wedge.bin(g)
    with pytest.raises(wedge.WedgeError) as e:
        wedge.sample(g, b, seed=1, k_per_bin=10, k_global=10, flags=wedge.FLAG_ROUNDING, first_sample=5)
    assert e.value.status == 1
    r = wedge.Requests([{"graph": g, "bins": b, "seed": 1, "k_per_bin": 10, "k_global": 10,
                         "flags": wedge.FLAG_ROUNDING}])
    with pytest.raises(wedge.WedgeError) as e:
        wedge.sample_batch(r)
    assert e.value.status == 1


def test_profile_and_repeatable():
    src, dst = graphgen.kronecker_host(12, seed=2)
    g = wedge.graph_build(src, dst, 1 << 12)
    b = wedge.bin(g)
    wedge.profile_enable(False)
    wedge.profile_reset()
    a = wedge.sample(g, b, seed=4, k_per_bin=50_000, flags=wedge.FLAG_ROUNDING | wedge.FLAG_NO_GLOBAL)
    prof = wedge.profile_read()
    for name in ("round_alloc", "scan_round_counts", "round_bin_base", "round_draw"):
        assert prof[name]["launches"] == 1
    assert "sample_closure" not in prof
    c = wedge.sample(g, b, seed=4, k_per_bin=50_000, flags=wedge.FLAG_ROUNDING | wedge.FLAG_NO_GLOBAL)
    assert np.array_equal(a.counts_matrix(), c.counts_matrix())
