"""Checkpoint and resume of the graph handle (wedge_graph_from_csr).

A CSR saved from a built graph (to host memory or a file) becomes a graph
again without the sort, is checked row by row on the device, and samples
exactly like the original; sampling resumes from any sample index
(first_sample), so a run split at a checkpoint gives the uninterrupted
run's counts. A damaged CSR (an unsorted row, a self-loop, an id out of
range, offsets that do not end at n_adj) is refused with EINVAL.
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


def _graph(scale=12, seed=3):
    src, dst = graphgen.kronecker_host(scale, seed=seed)
    return src, dst, 1 << scale


def test_saved_csr_resumes_exactly(tmp_path):
    src, dst, n = _graph()
    g = wedge.graph_build(torch.as_tensor(src).cuda(), torch.as_tensor(dst).cuda(), n)
    b = wedge.bin(g)
    ref = wedge.sample(g, b, seed=5, k_per_bin=4000, k_global=6000)
    path = str(tmp_path / "g.npz")
    wedge.graph_save(g, path)
    off, adj, deg = g.csr_numpy()
    gi0 = g.info()
    b.free()
    g.free()
    for g2 in (wedge.graph_load(path),  # from a file (host arrays)
               wedge.graph_from_csr(torch.as_tensor(off).cuda(), torch.as_tensor(adj).cuda(), n)):  # device arrays
        off2, adj2, deg2 = g2.csr_numpy()
        assert np.array_equal(off2, off) and np.array_equal(adj2, adj) and np.array_equal(deg2, deg)
        assert g2.info().max_degree == gi0.max_degree and g2.info().n_adj == gi0.n_adj
        b2 = wedge.bin(g2)
        c = wedge.sample(g2, b2, seed=5, k_per_bin=4000, k_global=6000)
        assert np.array_equal(c.counts_matrix(), ref.counts_matrix()) and c.closed_global == ref.closed_global
        # a run split at sample 2500: the two halves add up to the whole run
        c1 = wedge.sample(g2, b2, seed=5, k_per_bin=2500, k_global=2500)
        c2 = wedge.sample(g2, b2, seed=5, k_per_bin=1500, k_global=3500, first_sample=2500)
        assert np.array_equal(c1.counts_matrix()[:, 1:] + c2.counts_matrix()[:, 1:], ref.counts_matrix()[:, 1:])
        assert c1.closed_global + c2.closed_global == ref.closed_global
        b2.free()
        g2.free()
    # the oracle on the reloaded CSR
    ro, ra = oracle.csr(src, dst, n)
    assert np.array_equal(ro, off) and np.array_equal(ra, adj)


def test_damaged_csr_is_refused():
    src, dst, n = _graph(10, 8)
    off, adj = oracle.csr(src, dst, n)
    row = int(np.argmax(np.diff(off)))  # a row with several entries
    a0 = int(off[row])
    cases = []
    bad = adj.copy(); bad[a0], bad[a0 + 1] = bad[a0 + 1], bad[a0]; cases.append((off, bad))     # unsorted row
    a1 = int(off[row + 1])
    bad = adj.copy(); bad[a0] = row; bad[a0:a1].sort(); cases.append((off, bad))             # a self-loop, row still ascending
    bad = adj.copy(); bad[int(off[-1]) - 1] = n; cases.append((off, bad))                    # an id out of range
    bad_off = off.copy(); bad_off[-1] += 2; cases.append((bad_off, adj))                     # off[n] != n_adj
    bad_off = off.copy(); bad_off[5], bad_off[6] = bad_off[6] + 1, bad_off[5]; cases.append((bad_off, adj))  # not monotone
    for o, a in cases:
        with pytest.raises(wedge.WedgeError) as e:
            wedge.graph_from_csr(o, a, n)
        assert e.value.status == 1
    g = wedge.graph_from_csr(off, adj, n)  # the undamaged one is accepted
    assert g.info().n_adj == adj.shape[0]
    g.free()
