"""The oracle's Philox4x32-10 (written from the published definition of
Salmon et al., SC 2011) against cuRAND's public implementation of the same
generator, run on the GPU: an independent pin of every random word the
oracle, and so the bit-exact device path, draws."""
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_matches_curand(tmp_path):
    exe = tmp_path / "philox_curand"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-o", str(exe),
                    os.path.join(HERE, "philox_curand.cu")], check=True)
    rng = np.random.default_rng(2026)
    n = 4096
    words = rng.integers(0, 2**32, (n, 6), dtype=np.uint64).astype(np.uint32)
    words[:64, :4] = np.arange(64)[:, None]        # small counters, as the samplers use
    words[64:128] = 0xFFFFFFFF                      # all ones
    words[128:192, 2:4] = [[5, 0], [5, 1]] * 32     # bin / tag words
    (tmp_path / "in.bin").write_bytes(words.tobytes())
    subprocess.run([str(exe), str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], check=True)
    got = np.frombuffer((tmp_path / "out.bin").read_bytes(), dtype=np.uint32).reshape(n, 4)
    for i in range(n):
        ref = oracle.philox4x32_10(words[i, :4], words[i, 4:])
        assert list(map(int, ref)) == list(map(int, got[i])), i
