"""WEDGE_FLAG_SORTED_CLOSURE (closure queries sorted, then checked in order,
after Alg. Phase 3b's join of wedges with the edge list) on GB300: the same
samples as the inline check, so the per-bin tallies must equal the oracle's
bit for bit, for any bins, budgets and sample offsets.
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


def _compare(src, dst, n, tau, omega, seed, k, k_bin=None, k_global=0, first=0):
    g = wedge.graph_build(src, dst, n)
    b = wedge.bin(g, tau=tau, omega=omega)
    flags = wedge.FLAG_SORTED_CLOSURE | (0 if k_global else wedge.FLAG_NO_GLOBAL)
    got = wedge.sample(g, b, seed=seed, k_per_bin=k, k_global=k_global, flags=flags, k_bin=k_bin,
                       first_sample=first)
    inline = wedge.sample(g, b, seed=seed, k_per_bin=k, k_global=k_global,
                          flags=0 if k_global else wedge.FLAG_NO_GLOBAL, k_bin=k_bin, first_sample=first)
    assert np.array_equal(got.counts_matrix(), inline.counts_matrix())
    off, adj = oracle.csr(src, dst, n)
    ref = oracle.sample(off, adj, tau, omega, seed, k, k_global, k_bins=k_bin, first=first)
    assert np.array_equal(got.counts_matrix(), ref["counts"])
    if k_global:
        assert got.closed_global == int(ref["glob"][1]) and np.array_equal(got.stats, ref["stats"])
    return got


@pytest.mark.parametrize("scale,tau,omega,k", [(10, 1, 2, 3000), (12, 1, 2, 100_003), (12, 2, 2, 20_000),
                                               (11, 3, 5, 7777), (14, 1, 2, 1)])
def test_kronecker(scale, tau, omega, k):
    src, dst = graphgen.kronecker_host(scale, seed=scale + 3)
    _compare(src, dst, 1 << scale, tau, omega, 70 + scale, k, k_global=999)


def test_noisy_and_chunglu_with_offsets():
    src, dst = graphgen.kronecker_host(13, seed=2, noise=0.1)
    _compare(src, dst, 1 << 13, 1, 2, 5, 50_000, first=12345)
    n = 1 << 14
    prefix, m = graphgen.chunglu_weights(n, 2.0, 20.0)
    s, d = graphgen.chunglu_host(prefix, m, seed=4)
    _compare(s, d, n, 1, 2, 6, 200_000)


def test_budgets_per_bin():
    src, dst = graphgen.kronecker_host(12, seed=9)
    g = wedge.graph_build(src, dst, 1 << 12)
    nb = wedge.bin(g).info().n_bins
    kb = np.zeros(nb, np.uint64)
    kb[3::3] = 4000
    kb[nb - 1] = 100_000
    _compare(src, dst, 1 << 12, 1, 2, 8, 0, k_bin=kb)


def test_key_width_limit_and_exclusive_flags():
    src, dst = graphgen.kronecker_host(10, seed=1)
    g = wedge.graph_build(src, dst, (1 << 31) - 1)  # 31 id bits: 62 + payload > 64
    b = wedge.bin(g)
    with pytest.raises(wedge.WedgeError) as e:
        wedge.sample(g, b, seed=1, k_per_bin=10, flags=wedge.FLAG_SORTED_CLOSURE | wedge.FLAG_NO_GLOBAL)
    assert e.value.status == 1
    g2 = wedge.graph_build(src, dst, 1 << 10)
    b2 = wedge.bin(g2)
    with pytest.raises(wedge.WedgeError):
        wedge.sample(g2, b2, seed=1, k_per_bin=10, flags=wedge.FLAG_SORTED_CLOSURE | wedge.FLAG_ROUNDING)


def test_launches():
    src, dst = graphgen.kronecker_host(12, seed=2)
    g = wedge.graph_build(src, dst, 1 << 12)
    b = wedge.bin(g)
    wedge.profile_enable(False)
    wedge.profile_reset()
    wedge.sample(g, b, seed=4, k_per_bin=50_000, flags=wedge.FLAG_SORTED_CLOSURE | wedge.FLAG_NO_GLOBAL)
    prof = wedge.profile_read()
    assert prof["sorted_keys"]["launches"] == 1 and prof["sorted_closure"]["launches"] == 1
    assert "sample_closure" not in prof
