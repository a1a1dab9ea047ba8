"""Noisy Stochastic Kronecker generator (Sec. 5.1: noise parameter 0.1) — CPU.

Per level l the generator matrix is [a - 2 mu a/(a+d), b + mu; c + mu,
d - 2 mu d/(a+d)] with mu uniform in [-noise, noise] (Seshadhri, Pinar and
Kolda's noisy SKG). The checks recover each level's matrix from its integer
thresholds and test the relations between its entries, the per-level
quadrant frequencies of generated edges, and the smoothing of the degree
distribution that motivates the noise.
"""
import numpy as np

import graphgen
import oracle

A, B, C = graphgen.RMAT_A, graphgen.RMAT_B, graphgen.RMAT_C
D = 1.0 - A - B - C


def _matrices(th):
    t = th.astype(np.float64) / 2.0**32
    a = t[:, 0]
    b = t[:, 1] - t[:, 0]
    c = t[:, 2] - t[:, 1]
    d = 1.0 - t[:, 2]
    return a, b, c, d


def test_zero_noise_is_the_plain_generator():
    th = graphgen.rmat_levels(14, 0.0)
    assert (th == th[0]).all()
    s0, d0 = graphgen.kronecker_host(14)
    import ctypes  # noqa: F401 - the levels entry point through the same library
    src = np.empty(16 << 14, np.int32)
    dst = np.empty(16 << 14, np.int32)
    rc = graphgen._H().graphgen_kronecker_levels_host(14, 0, 16 << 14, graphgen._ptr(th), 1, 1, graphgen._ptr(src),
                                                      graphgen._ptr(dst))
    assert rc == 0 and np.array_equal(src, s0) and np.array_equal(dst, d0)


def test_level_matrices_follow_the_noise_rule():
    th = graphgen.rmat_levels(30, 0.1, seed=3)
    a, b, c, d = _matrices(th)
    mu_b, mu_c = b - B, c - C
    tol = 4.0 / 2.0**32  # threshold quantisation
    assert np.all(np.abs(mu_b - mu_c) <= tol)                   # both off-diagonals move by mu
    assert np.all(np.abs(mu_b) <= 0.1 + tol)                    # mu in [-0.1, 0.1]
    assert np.all(np.abs(a - (A - 2 * mu_b * A / (A + D))) <= 2 * tol)
    assert np.all(np.abs(d - (D - 2 * mu_b * D / (A + D))) <= 2 * tol)
    assert np.abs(mu_b).max() > 0.05 and np.std(mu_b) > 0.03    # the noise is really there
    assert not np.array_equal(th, graphgen.rmat_levels(30, 0.1, seed=4))  # and depends on the seed


def test_bad_noise_is_rejected():
    import pytest
    with pytest.raises(ValueError):
        graphgen.rmat_levels(10, 0.2)   # more than b = 0.19
    with pytest.raises(ValueError):
        graphgen.rmat_levels(10, -0.1)


def test_quadrant_frequencies_per_level():
    """Unpermuted edges: bit l of (u, v) falls in each quadrant with that level's probabilities."""
    S = 12
    th = graphgen.rmat_levels(S, 0.1, seed=9)
    a, b, c, d = _matrices(th)
    src, dst = graphgen.kronecker_host(S, n_edges=300000, permute=False, seed=9, noise=0.1)
    for level in range(S):
        sh = S - 1 - level
        bu = (src >> sh) & 1
        bv = (dst >> sh) & 1
        f = [np.mean((bu == 0) & (bv == 0)), np.mean((bu == 0) & (bv == 1)),
             np.mean((bu == 1) & (bv == 0)), np.mean((bu == 1) & (bv == 1))]
        for got, want in zip(f, (a[level], b[level], c[level], d[level])):
            assert abs(got - want) < 0.006, (level, f, (a[level], b[level], c[level], d[level]))


def test_noise_smooths_the_degree_distribution():
    """Plain SKG degree bins oscillate (Sec. 5.1 and the cited analysis); with noise 0.1 the counts per
    bin (tau = 2, omega = 2) fall off without the large up-and-down swings."""
    def swings(noise):
        s, d = graphgen.kronecker_host(16, noise=noise, seed=5)
        off, _ = oracle.csr(s, d, 1 << 16)
        deg = oracle.degrees(off)
        h = np.bincount([oracle.bin_id(int(x), 2, 2) for x in deg if x > 0]).astype(np.float64)
        h = h[3:np.nonzero(h)[0].max() + 1]
        r = np.log((h[1:] + 1) / (h[:-1] + 1))
        return int(np.sum((r[1:] > 0.5) & (r[:-1] < -0.5)) + np.sum((r[1:] < -0.5) & (r[:-1] > 0.5)))
    assert swings(0.0) >= 2 and swings(0.1) == 0
