"""Continuous-batching server (wedge_server_*) on GB300.

Requests of different eps arrive from several threads while earlier ones
run; each result must equal the same request run alone (wedge_sample on the
same graph), and the oracle for a subset. Admission evicts idle graphs
least-recently used first and rejects uploads that cannot fit.
"""
import threading

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


def _edges(i):
    if i % 2 == 0:
        scale = 9 + i // 2
        s, d = graphgen.kronecker_host(scale, seed=50 + i)
        return s, d, 1 << scale
    n = 1 << (10 + i // 2)
    prefix, m = graphgen.chunglu_weights(n, 2.0 + 0.1 * i, 12.0 + 4 * i)
    s, d = graphgen.chunglu_host(prefix, m, seed=60 + i)
    return s, d, n


def test_results_same_alone_and_in_the_mix():
    graphs = [_edges(i) for i in range(6)]
    srv = wedge.Server(slots=3)
    ids = []
    for i, (s, d, n) in enumerate(graphs):
        src = s if i < 3 else torch.as_tensor(s).cuda()  # host and device uploads
        dst = d if i < 3 else torch.as_tensor(d).cuda()
        ids.append(srv.add_graph(src, dst, n))
    rng = np.random.default_rng(7)
    eps_choices = [0.05, 0.02, 0.01]
    plan = [(int(rng.integers(0, 6)), int(rng.integers(1, 1 << 40)), float(rng.choice(eps_choices)))
            for _ in range(160)]
    tickets = [None] * len(plan)
    results = [None] * len(plan)

    def submitter(part):
        for j in part:
            gi, seed, eps = plan[j]
            tickets[j] = srv.submit(ids[gi], seed, eps=eps, delta=0.001)

    threads = [threading.Thread(target=submitter, args=(range(t, len(plan), 4),)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for j in range(len(plan)):
        results[j] = srv.wait(tickets[j])
    st = srv.stats()
    assert st["completed"] == len(plan)
    assert st["p50_us"] > 0 and st["p99_us"] >= st["p50_us"]
    assert 1 <= st["batches"] <= len(plan)
    assert st["resident_graphs"] == 6

    alone = []
    for s, d, n in graphs:
        g = wedge.graph_build(s, d, n)
        alone.append((g, wedge.bin(g, tau=1, omega=2)))
    for j, (gi, seed, eps) in enumerate(plan):
        c, tm = results[j]
        g, b = alone[gi]
        ref = wedge.sample(g, b, seed=seed, eps=eps, delta=0.001)
        assert np.array_equal(c.counts_matrix(), ref.counts_matrix())
        assert c.closed_global == ref.closed_global and np.array_equal(c.stats, ref.stats)
        assert tm["done_us"] >= tm["dispatch_us"] >= tm["submit_us"] and tm["batch_requests"] >= 1
    # a few against the oracle
    for j in range(0, len(plan), 40):
        gi, seed, eps = plan[j]
        s, d, n = graphs[gi]
        off, adj = oracle.csr(s, d, n)
        k = oracle.hoeffding_k(eps, 0.001)
        ref = oracle.sample(off, adj, 1, 2, seed, k, k)
        c, _ = results[j]
        assert np.array_equal(c.counts_matrix(), ref["counts"]) and c.closed_global == int(ref["glob"][1])
    srv.close()


def test_admission_evicts_idle_graphs_lru():
    s, d, n = _edges(2)  # Kronecker scale 10: 16,384 edges
    m = s.shape[0]
    resident_est = 8 * m + 24 * n + 16                                   # what a built graph keeps
    need = resident_est + 2 * 8 * 2 * m + 2 * m // 16 + 8 * m + 16 * n  # plus its build scratch
    # room for one resident graph and an upload, but not for two and an upload
    srv = wedge.Server(hbm_budget_bytes=need + int(1.5 * resident_est), slots=2)
    a = srv.add_graph(s, d, n)
    b = srv.add_graph(s, d, n)
    c = srv.add_graph(s, d, n)  # evicts the least recently used idle graph (a)
    st = srv.stats()
    assert st["evictions"] >= 1 and st["resident_graphs"] <= 2
    with pytest.raises(wedge.WedgeError) as e:
        srv.submit(a, 1, k_per_bin=100, k_global=100)
    assert e.value.status == 1
    t = srv.submit(c, 1, k_per_bin=100, k_global=100)
    cnt, _ = srv.wait(t)
    assert cnt.k_global == 100
    big_s, big_d = graphgen.kronecker_host(14)
    with pytest.raises(wedge.WedgeError) as e:  # larger than the whole budget
        srv.add_graph(big_s, big_d, 1 << 14)
    assert e.value.status == 2
    assert srv.stats()["rejected_uploads"] >= 1
    srv.remove_graph(c)
    with pytest.raises(wedge.WedgeError):
        srv.remove_graph(c)
    del b
    srv.close()


def test_many_small_requests_batch_together():
    s, d, n = _edges(4)
    srv = wedge.Server(slots=1)
    gid = srv.add_graph(s, d, n)
    # occupy the only slot, then queue many small requests behind it
    first = srv.submit(gid, 1, k_per_bin=200000, k_global=200000)
    tickets = [srv.submit(gid, 100 + i, k_per_bin=500, k_global=500) for i in range(64)]
    srv.wait(first)
    sizes = [srv.wait(t)[1]["batch_requests"] for t in tickets]
    assert max(sizes) > 1  # requests that arrived during the first batch were admitted together
    srv.close()


def _request_samples(b, k_bin, k_glob):
    """A request's size as the server counts it: the per-bin budget over the
    bins with wedges, plus the global budget."""
    bi = b.info()
    return k_bin * int((np.array(bi.p_b[: bi.n_bins], np.uint64) != 0).sum()) + k_glob


def test_admission_control_refuses_when_queue_is_full():
    s, d, n = _edges(4)
    g = wedge.graph_build(s, d, n)
    b = wedge.bin(g, tau=1, omega=2)
    size = _request_samples(b, 50000, 50000)
    # the queue may hold three such requests; one more waits in the only slot
    srv = wedge.Server(slots=1, max_queued_samples=3 * size)
    gid = srv.add_graph(s, d, n)
    tickets, refused = [], 0
    for i in range(40):  # submitted far faster than one slot drains them
        try:
            tickets.append((srv.submit(gid, 1000 + i, k_per_bin=50000, k_global=50000), 1000 + i))
        except wedge.WedgeError as e:
            assert e.status == wedge.EBUSY
            refused += 1
    st = srv.stats()
    assert refused >= 1 and st["rejected_requests"] == refused
    assert st["queued_samples"] <= 3 * size
    for t, seed in tickets:  # what was admitted is exact
        c, _ = srv.wait(t)
        ref = wedge.sample(g, b, seed=seed, k_per_bin=50000, k_global=50000)
        assert np.array_equal(c.counts_matrix(), ref.counts_matrix()) and c.closed_global == ref.closed_global
    assert srv.stats()["queued_samples"] == 0
    srv.close()
    b.free()
    g.free()


def test_batches_respect_the_sample_cap_and_large_requests_do_not_pair():
    s, d, n = _edges(4)
    g = wedge.graph_build(s, d, n)
    b = wedge.bin(g, tau=1, omega=2)
    small = _request_samples(b, 1000, 1000)
    large = _request_samples(b, 400000, 400000)
    srv = wedge.Server(slots=2, max_batch_samples=8 * small, gpu_filling_samples=large)
    gid = srv.add_graph(s, d, n)
    big = [srv.submit(gid, 1 + i, k_per_bin=400000, k_global=400000) for i in range(3)]
    little = [srv.submit(gid, 100 + i, k_per_bin=1000, k_global=1000) for i in range(48)]
    big_t = [srv.wait(t)[1] for t in big]
    little_t = [srv.wait(t)[1] for t in little]
    # no batch holds more than 8 small requests' samples (a large one alone)
    assert all(tm["batch_requests"] == 1 for tm in big_t)
    assert all(tm["batch_requests"] <= 8 for tm in little_t)
    # two large requests never ran at the same time
    spans = sorted((tm["dispatch_us"], tm["done_us"]) for tm in big_t)
    for (d0, e0), (d1, e1) in zip(spans, spans[1:]):
        assert d1 >= e0 - 50.0  # dispatched only after the previous large one finished (poll granularity)
    # small requests overtook the queued large ones
    assert min(tm["done_us"] for tm in little_t) < max(tm["done_us"] for tm in big_t)
    srv.close()
    b.free()
    g.free()
