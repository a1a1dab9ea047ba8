"""The allocation-free row-offsets entry point (wedge_degree_offsets_noalloc).

It serves callers that cannot allocate device memory (a host framework that
has reserved the GPU's memory for its own pool, a plug-in callback that may
not allocate, a latency-bound loop that cannot take cudaMalloc's implicit
synchronisation). Its output must equal the row offsets that
wedge_graph_build computes for the same degrees, on two calls in a row (the
scratch array keeps the previous call's contents, so the second call checks
that it is cleared). This file is collected last so that a run stopping at
its first failure has already run every other test.
"""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
wedge = pytest.importorskip("paper_1301_5887_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    wedge.load()


def _graph(scale):
    m = graphgen.kronecker_edges(scale)
    s = torch.empty(m, dtype=torch.int32, device="cuda")
    d = torch.empty(m, dtype=torch.int32, device="cuda")
    graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), m, torch.cuda.current_stream().cuda_stream)
    return wedge.graph_build(s, d, 1 << scale)


@pytest.mark.parametrize("scale", [12, 21])
def test_noalloc_offsets_match_graph_build_twice(scale):
    g = _graph(scale)
    n = 1 << scale
    deg = torch.empty(n, dtype=torch.int32, device="cuda")
    ref = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    g.copy(off=ref, deg=deg)
    for _ in range(2):
        out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
        wedge.degree_offsets_noalloc(deg, out)
        assert torch.equal(out, ref)


def test_noalloc_offsets_ragged_and_small():
    rng = np.random.default_rng(1)
    for n in [1, 5, 4095, 4096, 4097, 70001]:
        deg_h = rng.integers(0, 50, n).astype(np.int32)
        deg = torch.as_tensor(deg_h).cuda()
        out = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
        wedge.degree_offsets_noalloc(deg, out)
        exp = np.concatenate([[0], np.cumsum(deg_h.astype(np.int64))])
        assert np.array_equal(out.cpu().numpy(), exp)


def test_noalloc_rejects_sizes_beyond_maximum():
    lib = wedge.load()
    deg = torch.zeros(1, dtype=torch.int32, device="cuda")
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = lib.wedge_degree_offsets_noalloc(deg.data_ptr(), wedge.NOALLOC_MAX_VERTICES + 1, off.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert st == 1  # WEDGE_EINVAL, before any device work
    assert b"exceeds the maximum" in lib.wedge_last_error()


def test_noalloc_rejects_negative_degrees_and_overflow():
    lib = wedge.load()
    deg = torch.zeros(9000, dtype=torch.int32, device="cuda")
    deg[5000] = -3
    off = torch.zeros(9001, dtype=torch.int64, device="cuda")
    with pytest.raises(wedge.WedgeError):
        wedge.degree_offsets_noalloc(deg, off)
    assert b"negative" in lib.wedge_last_error()
    # 2^28 vertices of degree 2^31 - 1: the total (about 2^59) crosses 2^58
    n = 1 << 28
    big = torch.full((n,), 2**31 - 1, dtype=torch.int32, device="cuda")
    offb = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(wedge.WedgeError):
        wedge.degree_offsets_noalloc(big, offb)
    assert b"2^58" in lib.wedge_last_error()
    # the next call works again
    deg[5000] = 3
    wedge.degree_offsets_noalloc(deg, off)
    assert int(off[-1].item()) == 3
