"""Batched persistent sampling (wedge_batch_*, wedge_autotune) on GB300.

A mix of Kronecker and Chung-Lu graphs with per-bin budgets drawn
log-uniformly; every request's counts must equal the oracle's bit for bit
and equal a plain wedge_sample call, for every mapping, block size and tile
size, on repeated (CUDA-graph) launches and in any request order.
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


def _kron(scale, seed):
    m = graphgen.kronecker_edges(scale)
    s = torch.empty(m, dtype=torch.int32, device="cuda")
    d = torch.empty(m, dtype=torch.int32, device="cuda")
    graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), m, torch.cuda.current_stream().cuda_stream,
                              seed=seed)
    hs, hd = graphgen.kronecker_host(scale, seed=seed)
    return wedge.graph_build(s, d, 1 << scale), oracle.csr(hs, hd, 1 << scale)


def _chunglu(n, gamma, mean_deg, seed):
    prefix, m = graphgen.chunglu_weights(n, gamma, mean_deg)
    pd = torch.as_tensor(prefix.view(np.int64)).cuda()
    s = torch.empty(m, dtype=torch.int32, device="cuda")
    d = torch.empty(m, dtype=torch.int32, device="cuda")
    graphgen.chunglu_device(pd.data_ptr(), n, s.data_ptr(), d.data_ptr(), m, seed,
                            stream_ptr=torch.cuda.current_stream().cuda_stream)
    hs, hd = graphgen.chunglu_host(prefix, m, seed)
    assert np.array_equal(s.cpu().numpy(), hs) and np.array_equal(d.cpu().numpy(), hd)
    return wedge.graph_build(s, d, n), oracle.csr(hs, hd, n)


@pytest.fixture(scope="module")
def mix():
    rng = np.random.default_rng(2024)
    graphs = []
    for i, scale in enumerate([8, 9, 10, 11, 12, 13]):
        graphs.append(_kron(scale, seed=100 + i))
    for i, (lg, gamma, dbar) in enumerate([(10, 2.0, 8.0), (11, 2.3, 30.0), (12, 2.6, 64.0), (10, 2.1, 16.0)]):
        graphs.append(_chunglu(1 << lg, gamma, dbar, seed=200 + i))
    reqs = []
    for i, (g, (off, adj)) in enumerate(graphs):
        b = wedge.bin(g, tau=1, omega=2)
        nb = b.info().n_bins
        k_bin = np.exp(rng.uniform(np.log(1e3), np.log(2e4), nb)).astype(np.uint64)
        k_glob = int(np.exp(rng.uniform(np.log(1e3), np.log(2e4))))
        reqs.append({"graph": g, "bins": b, "seed": 1000 + i, "k_bin": k_bin, "k_global": k_glob,
                     "off": off, "adj": adj})
    return reqs


def _oracle_counts(r):
    return oracle.sample(r["off"], r["adj"], 1, 2, r["seed"], 0, r["k_global"], k_bins=r["k_bin"])


def _same(c, ref):
    assert c.n_bins == ref["counts"].shape[0]
    assert np.array_equal(c.counts_matrix(), ref["counts"])
    assert c.k_global == int(ref["glob"][0]) and c.closed_global == int(ref["glob"][1])
    assert np.array_equal(c.stats, ref["stats"])


def test_batch_matches_oracle_and_plain(mix):
    out = wedge.sample_batch(wedge.Requests(mix))
    for r, c in zip(mix, out):
        _same(c, _oracle_counts(r))
        p = wedge.sample(r["graph"], r["bins"], seed=r["seed"], k_global=r["k_global"], k_bin=r["k_bin"])
        assert np.array_equal(c.counts_matrix(), p.counts_matrix()) and c.closed_global == p.closed_global


@pytest.mark.parametrize("cfg", [
    {"block_threads": 128, "samples_per_tile": 1024},
    {"block_threads": 512, "samples_per_tile": 4096},
    {"mapping_small": 2, "mapping_medium": 2, "mapping_large": 2, "block_threads": 256, "samples_per_tile": 512},
    {"mapping_small": 2, "mapping_medium": 1, "mapping_large": 2, "block_threads": 128, "samples_per_tile": 3000},
])
def test_batch_invariant_to_launch_shape(mix, cfg):
    ref = wedge.sample_batch(wedge.Requests(mix))
    got = wedge.sample_batch(wedge.Requests(mix), cfg=cfg)
    for a, b in zip(ref, got):
        assert np.array_equal(a.counts_matrix(), b.counts_matrix())
        assert a.closed_global == b.closed_global and np.array_equal(a.stats, b.stats)


def test_batch_order_and_replay(mix):
    ref = wedge.sample_batch(wedge.Requests(mix))
    order = list(reversed(range(len(mix))))
    batch = wedge.Batch(wedge.Requests([mix[i] for i in order]))
    info = batch.info()
    assert info["tiles"] > 0 and info["grid"] > 0
    for _ in range(3):  # graph replays start from cleared counters
        batch.launch()
        got = batch.results()
        for j, i in enumerate(order):
            assert np.array_equal(got[j].counts_matrix(), ref[i].counts_matrix())
            assert got[j].closed_global == ref[i].closed_global
    batch.free()


@pytest.mark.parametrize("spt", [512, 1000, 4096])
def test_batch_tiles_are_per_stream(mix, spt):
    """The tile list is implicit: one stream per nonempty bin with a budget
    (and the global stream), each cut into ceil(k / samples_per_tile) tiles;
    the counts stay exact for tile sizes that do not divide the budgets."""
    batch = wedge.Batch(wedge.Requests(mix), cfg={"samples_per_tile": spt})
    info = batch.info()
    batch.launch()
    got = batch.results()
    batch.free()
    streams = tiles = 0
    for r in mix:
        bi = r["bins"].info()
        for k in range(2, bi.n_bins):
            if bi.p_b[k] > 0 and int(r["k_bin"][k]) > 0:
                streams += 1
                tiles += -(-int(r["k_bin"][k]) // spt)
        if bi.p_total > 0 and r["k_global"] > 0:
            streams += 1
            tiles += -(-int(r["k_global"]) // spt)
    assert info["streams"] == streams and info["tiles"] == tiles
    ref = wedge.sample_batch(wedge.Requests(mix))
    for a, b in zip(got, ref):
        assert np.array_equal(a.counts_matrix(), b.counts_matrix()) and a.closed_global == b.closed_global


def test_batch_records_match_plain(mix):
    r = mix[3]
    rec_b = torch.zeros((r["k_global"], 8), dtype=torch.int32, device="cuda")
    rec_p = torch.zeros((r["k_global"], 8), dtype=torch.int32, device="cuda")
    item = dict(r)
    item["records"] = rec_b
    wedge.sample_batch(wedge.Requests([item]), cfg={"mapping_small": 2, "mapping_medium": 2, "mapping_large": 2})
    wedge.sample(r["graph"], r["bins"], seed=r["seed"], k_global=r["k_global"], k_bin=r["k_bin"], records=rec_p)
    assert torch.equal(rec_b, rec_p)
    ref = oracle.sample(r["off"], r["adj"], 1, 2, r["seed"], 0, r["k_global"], records=True, k_bins=r["k_bin"])
    assert np.array_equal(rec_b.cpu().numpy(), ref["records"])


def test_autotune_config_is_valid_and_exact(mix):
    reqs = wedge.Requests(mix)
    cfg = wedge.autotune(reqs)
    d = cfg.as_dict()
    assert d["block_threads"] in (128, 256, 512) and d["samples_per_tile"] in (1024, 2048, 4096)
    for k in ("mapping_small", "mapping_medium", "mapping_large"):
        assert d[k] in (1, 2)
    assert wedge.autotune(reqs).as_dict() == d  # cached
    ref = wedge.sample_batch(wedge.Requests(mix))
    got = wedge.sample_batch(reqs, cfg=cfg)
    for a, b in zip(ref, got):
        assert np.array_equal(a.counts_matrix(), b.counts_matrix())


def test_batch_edge_cases(mix):
    assert wedge.sample_batch(wedge.Requests([])) == []
    r = dict(mix[0])
    r["flags"] = wedge.FLAG_NO_BINS
    c = wedge.sample_batch(wedge.Requests([r]))[0]
    assert int(c.k_b.sum()) == 0 and c.k_global == r["k_global"]
    bad = dict(mix[0])
    bad["bins"] = mix[1]["bins"]
    with pytest.raises(wedge.WedgeError) as e:
        wedge.sample_batch(wedge.Requests([bad]))
    assert e.value.status == 1
    with pytest.raises(wedge.WedgeError):
        wedge.sample_batch(wedge.Requests(mix[:1]), cfg={"block_threads": 100})


def test_autotune_scaled_probe_for_large_batches(mix):
    """Requests totalling more than 1.5e9 samples are tuned on budgets and
    tile sizes scaled down by the same factor; the chosen shape is one of the
    candidates at full scale and the batch still equals plain calls."""
    big = []
    for r in mix:
        item = dict(r)
        item["k_bin"] = np.zeros_like(r["k_bin"])
        item["k_global"] = 200_000_000
        big.append(item)
    cfg = wedge.autotune(wedge.Requests(big))
    d = cfg.as_dict()
    assert d["block_threads"] in (128, 256, 512) and d["samples_per_tile"] in (1024, 2048, 4096)
    got = wedge.sample_batch(wedge.Requests(big), cfg=cfg)
    for r, c in zip(big, got):
        p = wedge.sample(r["graph"], r["bins"], seed=r["seed"], k_global=r["k_global"], k_bin=r["k_bin"])
        assert c.k_global == p.k_global == r["k_global"] and c.closed_global == p.closed_global
        assert np.array_equal(c.stats, p.stats)
