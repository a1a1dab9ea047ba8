"""The C-ABI library loads without a GPU, exports every declared symbol, and
its pure-host entry points (budget, estimates, status strings) agree with the
oracle. No device computation runs here."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT

import paper_1301_5887_gb300 as wedge
from paper_1301_5887_gb300 import build as pkg_build

HEADER = os.path.join(ROOT, "include", "wedge.h")


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return wedge.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(wedge_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_binding_exports():
    assert sorted(wedge.EXPORTS) == declared_functions()


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", wedge.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(wedge_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # nothing else leaks out of the library under a wedge_ name
    assert exported == set(declared_functions())


def test_abi_struct_sizes_match(lib):
    sizes = (ctypes.c_uint64 * 16)()
    n = lib.wedge_abi_sizes(sizes, 16)
    assert n == len(wedge._STRUCTS)
    assert [int(sizes[i]) for i in range(n)] == [ctypes.sizeof(S) for S in wedge._STRUCTS]


def test_status_strings(lib):
    for code, name in wedge.STATUS.items():
        assert lib.wedge_status_str(code).decode() == name
    assert lib.wedge_version() >= 0x000100


def test_hoeffding_matches_oracle(lib):
    import oracle
    for eps, delta in [(0.002, 0.001), (0.01, 0.001), (0.005, 0.001), (0.05, 0.001), (0.1, 0.5), (0.3, 0.01)]:
        assert wedge.hoeffding_k(eps, delta) == oracle.hoeffding_k(eps, delta)
    assert wedge.hoeffding_k(0.0, 0.1) == 0 and wedge.hoeffding_k(0.1, 1.0) == 0


def _counts_from(counts_mat, p_b, glob, stats=None):
    c = wedge.CountsStruct()
    nb = counts_mat.shape[0]
    c.n_bins = nb
    for b in range(nb):
        c.k_b[b] = int(counts_mat[b, 0])
        for q in range(4):
            c.q[b][q] = int(counts_mat[b, 1 + q])
        c.p_b[b] = int(p_b[b])
    c.p_total = int(sum(int(x) for x in p_b))
    c.k_global, c.closed_global = int(glob[0]), int(glob[1])
    return wedge.Counts(c)


def test_estimate_matches_oracle_estimator(lib):
    """wedge_estimate (host FP64) vs the oracle's estimator on the same counts."""
    import graphgen
    import oracle
    from oracle.estimate import estimate as oracle_estimate
    src, dst = graphgen.kronecker_host(11)
    off, adj = oracle.csr(src, dst, 2048)
    r = oracle.sample(off, adj, 1, 2, seed=7, k_per_bin=3000, k_global=7000)
    bb = oracle.bins(off, 1, 2)
    for delta in [0.001, 0.05]:
        ref = oracle_estimate(bb["p_b"], r["counts"], r["glob"], delta)
        got = wedge.estimate(_counts_from(r["counts"], bb["p_b"], r["glob"]), delta)
        for key in ["c_hat", "t_hat", "c_hat_global", "t_hat_global", "eps_global"]:
            assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=0)
        for b in range(len(ref["c_b"])):
            assert got["c_b"][b] == pytest.approx(ref["c_b"][b], rel=1e-12, abs=0)
            assert got["t_b"][b] == pytest.approx(ref["t_b"][b], rel=1e-12, abs=0)
            assert got["eps_b"][b] == pytest.approx(ref["eps_b"][b], rel=1e-12, abs=0)


def test_estimate_rejects_bad_args(lib):
    c = _counts_from(np.zeros((3, 5), np.uint64), [0, 0, 0], [0, 0])
    with pytest.raises(wedge.WedgeError) as e:
        wedge.estimate(c, 0.0)
    assert e.value.status == 1
    with pytest.raises(wedge.WedgeError):
        wedge.estimate(c, 1.5)


def test_estimate_empty_bins_are_zero(lib):
    c = _counts_from(np.zeros((4, 5), np.uint64), [0, 0, 5, 0], [0, 0])
    e = wedge.estimate(c, 0.01)
    assert e["c_b"] == [0.0] * 4 and e["t_b"] == [0.0] * 4 and e["c_hat"] == 0.0
    assert not any(math.isnan(x) for x in e["eps_b"])


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib
    import paper_1301_5887_gb300 as mod
    monkeypatch.setattr(mod, "_SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mod, "_lib", None)
    with pytest.raises(ImportError):
        mod.load()
    importlib.reload(mod)


def test_no_oracle_import_in_product():
    """The product package never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_1301_5887_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.c" not in text and "liboracle" not in text, f


def test_noalloc_binding_checks_its_arguments(lib):
    """The allocation-free entry point's binding refuses host tensors, wrong
    dtypes, non-contiguous outputs and short outputs before any device call."""
    torch = pytest.importorskip("torch")
    deg = torch.zeros(8, dtype=torch.int32)
    off = torch.zeros(9, dtype=torch.int64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        wedge.degree_offsets_noalloc(deg, off)
    with pytest.raises(ValueError, match="CUDA tensor"):
        wedge.degree_offsets_noalloc(deg.numpy(), off.numpy())


def test_debug_build_exports_the_same_abi(lib):
    """libwedge_debug.so (bounds-checked) loads with the same struct sizes and
    exports exactly the symbols include/wedge.h declares."""
    dbg = wedge.load_debug()
    assert dbg.wedge_version() == lib.wedge_version()
    path = os.path.join(os.path.dirname(wedge.library_path()), "libwedge_debug.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    assert set(re.findall(r"\s[TW]\s+(wedge_\w+)", out)) == set(declared_functions())
