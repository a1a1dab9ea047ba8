"""Host-side arithmetic of bench.py, without a GPU.

Covers the algorithmic bytes behind roofline.frac, the rule that recorded
DRAM counters are used only on the sources they were taken on, and the
compact summary at the end of the JSON line.
"""
import json

import pytest

import bench


def test_sort_bytes_at_scale_28():
    # 7 forward passes over 2^32 keys and 3 transposed passes over the m
    # unique edges at 16 B per key (8 read, 8 written); the placing pass
    # reads 8 B and writes one 4-byte adjacency entry per key
    m = 4_236_157_710
    nkeys, launches, nbytes = bench.sort_sizes(1 << 32, 2 * m, 28)
    assert launches == 11
    assert nbytes == 16 * 7 * (1 << 32) + 16 * 3 * m + 12 * m
    assert abs(nbytes / 1e9 - 735.2) < 0.05
    assert nkeys == (7 * (1 << 32) + 4 * m) / 11


@pytest.mark.parametrize("b,pf,pt", [(1, 1, 1), (4, 1, 1), (5, 2, 1), (8, 2, 1), (9, 3, 2), (16, 4, 2),
                                     (17, 5, 3), (28, 7, 4), (31, 8, 4)])
def test_sort_pass_counts(b, pf, pt):
    # forward keys (min << b) | max have 2b significant bits, the transposed
    # sort runs over the b bits of the larger endpoint; 8-bit digits
    n, m = 1000, 300
    _, launches, nbytes = bench.sort_sizes(n, 2 * m, b)
    assert launches == pf + pt
    assert nbytes == 16 * pf * n + 16 * (pt - 1) * m + 12 * m


def test_algorithmic_bytes_per_kernel():
    z = {"n_edges": 100, "n_adj": 180, "n": 50, "n2": 40, "nkeys": 100, "sort_bytes": 1100, "sort_launches": 11}
    a = bench.ALG_BYTES
    assert a["sort_onesweep_pass"](z) == 100
    assert a["edge_histograms"](z) == 8 * 100  # the edges' two int32 endpoints, read once
    assert a["dedup_rows"](z) == 8 * 100 + 8 * 90  # keys in; a transposed key per unique edge out
    assert a["place_rows"](z) == 8 * 100 + 4 * 90  # keys in again; an int32 entry per unique edge out
    assert a["scan_degrees"](z) == 12 * 50  # int32 in, int64 out
    assert a["row_offsets"](z) == 36 * 50


def test_counters_are_used_only_on_the_sources_they_were_taken_on(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    entry = {"bytes_per_unit": 15.2, "source_hash": "current"}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"sort_onesweep_pass": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda kernel: "current")
    assert bench.ncu_figures("sort_onesweep_pass") == entry
    assert bench.ncu_figures("dedup_rows") is None  # never recorded
    monkeypatch.setattr(bench, "source_hash", lambda kernel: "edited")
    assert bench.ncu_figures("sort_onesweep_pass") is None  # the kernel changed since


def test_source_hash_follows_each_kernels_sources():
    h = bench.source_hash("sort_onesweep_pass")
    assert len(h) == 16 and h == bench.source_hash("sort_onesweep_pass")
    assert h != bench.source_hash("dedup_rows") != bench.source_hash("sample_closure")


def test_compact_summary():
    rates = [{"rate_per_s": 300.0,
              "served": {"p50_ms": 0.371, "p99_ms": 3.333, "gwedges_per_s": 1.8221, "rejected": 0},
              "plain": {"p50_ms": 0.722, "p99_ms": 4.191, "gwedges_per_s": 1.8201}}]
    batched = {"plain_gwedges_per_s": 5.626, "batched_gwedges_per_s": 8.247, "replay_gwedges_per_s": 8.34,
               "speedup": 1.466, "identical_to_plain": True, "roofline": {"frac": 0.2451}}
    out = bench.compact_summary(6.2259e-05, 263.7412, 3.3141, {"frac": 0.51934},
                                {"frac": 0.6713, "modelled_sectors_per_sample": 8.0},
                                {"ms_per_step": 681.63, "h2d_link_gbs": 80.43}, batched, {"rates": rates})
    assert out["ms_per_step"] == 263.74 and out["sort_pass_frac_of_copy_peak"] == 0.519
    assert out["e2e_ms_per_step"] == 681.6 and out["batched"]["identical_to_plain"] is True
    assert out["serving"][0]["served_p99_ms"] == 3.33 and out["serving"][0]["plain_p99_ms"] == 4.19
    # without the optional legs
    bare = bench.compact_summary(1.0, 2.0, 3.0, {"frac": 0.5}, {}, None, None, None)
    assert bare["e2e_ms_per_step"] is None and "batched" not in bare and "serving" not in bare
