"""Failure paths on the GPU, made without any device fault.

* A decoupled look-back wait that runs out: the library's scan kernel waits on
  a status word that nothing sets, with its poll limit lowered to a few
  thousand polls; the call returns WEDGE_ETIMEOUT within milliseconds and the
  library keeps working (the next build matches the oracle).
* An allocation refused on the host: the hook makes the k-th device
  allocation of an entry point fail, for every k in turn. Each call returns
  WEDGE_ENOMEM, produces no handle and leaves the pool's usage where it was
  (nothing leaks); once k passes the entry point's last allocation the call
  succeeds and gives the same result as without the hook.
"""
import time

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
wedge = pytest.importorskip("paper_1301_5887_gb300")

ENOMEM, ETIMEOUT = 2, 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    wedge.load()
    yield
    wedge.fail_next_allocation(-1)


def _kronecker(scale, seed=1):
    src, dst = graphgen.kronecker_host(scale, seed=seed)
    return src, dst, 1 << scale


def test_lookback_wait_runs_out_and_library_recovers():
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with pytest.raises(wedge.WedgeError) as e:
        wedge.force_lookback_timeout(4096)
    dt = time.perf_counter() - t0
    assert e.value.status == ETIMEOUT
    assert "gave up" in str(e.value)
    assert dt < 5.0  # a few thousand polls, not the production limit of about a second per wait
    # the context is intact: a build right after is exact
    src, dst, n = _kronecker(11)
    g = wedge.graph_build(torch.as_tensor(src).cuda(), torch.as_tensor(dst).cuda(), n)
    off, adj = oracle.csr(src, dst, n)
    goff, gadj, _ = g.csr_numpy()
    assert np.array_equal(goff, off) and np.array_equal(gadj, adj)
    g.free()
    with pytest.raises(wedge.WedgeError):
        wedge.force_lookback_timeout(0)  # out of range: EINVAL, nothing launched


def _used():
    torch.cuda.synchronize()
    return wedge.pool_used_bytes()


def _every_allocation_refused(call, check):
    """Refuse the k-th allocation of call() for k = 0, 1, ... until the call
    succeeds; every refused call must raise ENOMEM without leaking."""
    base = _used()
    k = 0
    while True:
        wedge.fail_next_allocation(k)
        try:
            out = call()
        except wedge.WedgeError as e:
            wedge.fail_next_allocation(-1)
            assert e.status == ENOMEM, (k, str(e))
            assert "refused by the test hook" in str(e)
            assert _used() == base, f"allocation {k}: pool usage {_used()} != {base} after ENOMEM"
            k += 1
            assert k < 200
            continue
        wedge.fail_next_allocation(-1)
        check(out)
        return k


def test_graph_build_enomem_at_every_allocation_device_input():
    src, dst, n = _kronecker(12)
    s, d = torch.as_tensor(src).cuda(), torch.as_tensor(dst).cuda()
    off, adj = oracle.csr(src, dst, n)

    def check(g):
        goff, gadj, _ = g.csr_numpy()
        assert np.array_equal(goff, off) and np.array_equal(gadj, adj)
        g.free()

    refused = _every_allocation_refused(lambda: wedge.graph_build(s, d, n), check)
    assert refused >= 8  # every buffer of the build was refused once


def test_graph_build_enomem_at_every_allocation_host_input():
    src, dst, n = _kronecker(12)
    hs, hd = torch.as_tensor(src).pin_memory(), torch.as_tensor(dst).pin_memory()
    off, adj = oracle.csr(src, dst, n)

    def check(g):
        goff, gadj, _ = g.csr_numpy()
        assert np.array_equal(goff, off) and np.array_equal(gadj, adj)
        g.free()

    refused = _every_allocation_refused(lambda: wedge.graph_build(hs, hd, n), check)
    assert refused >= 8


def test_bin_and_sample_enomem_at_every_allocation():
    src, dst, n = _kronecker(12)
    g = wedge.graph_build(torch.as_tensor(src).cuda(), torch.as_tensor(dst).cuda(), n)
    off, adj = oracle.csr(src, dst, n)
    ref_bins = oracle.bins(off, 1, 2)

    def check_bins(b):
        bi = b.info()
        assert bi.n_bins == len(ref_bins["n_b"])
        b.free()

    assert _every_allocation_refused(lambda: wedge.bin(g, tau=1, omega=2), check_bins) >= 2
    b = wedge.bin(g, tau=1, omega=2)
    ref = oracle.sample(off, adj, 1, 2, 7, 500, 5000)

    def check_counts(c):
        assert np.array_equal(c.counts_matrix(), ref["counts"])
        assert c.closed_global == int(ref["glob"][1])

    assert _every_allocation_refused(lambda: wedge.sample(g, b, seed=7, k_per_bin=500, k_global=5000),
                                     check_counts) >= 1
    b.free()
    g.free()
