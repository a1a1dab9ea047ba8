"""Sharded sampling across ranks, on CPU with the gloo backend (world size 2).

Each rank draws its contiguous share of every stream's sample indices (the
oracle stands in for a rank's GPU); one integer all-reduce of the counter
blocks must equal the unsharded counts exactly. Also the max-over-ranks
timing reduction used by bench.py.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1301_5887_gb300 import multi  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import graphgen
    import oracle
    from paper_1301_5887_gb300 import multi as m
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    src, dst = graphgen.kronecker_host(10)
    off, adj = oracle.csr(src, dst, 1024)
    k = 12345
    first, cnt = m.shard_range(k, rank, world)
    part = oracle.sample(off, adj, 1, 2, 77, cnt, cnt, first=first)
    cm, kg, cg, st = m.allreduce_counts(part["counts"], int(part["glob"][0]), int(part["glob"][1]), part["stats"])
    t = m.max_over_ranks(float(rank + 1))
    if rank == 0:
        full = oracle.sample(off, adj, 1, 2, 77, k, k)
        ok = (np.array_equal(cm, full["counts"]) and kg == int(full["glob"][0]) and cg == int(full["glob"][1])
              and np.array_equal(st, full["stats"]) and t == float(world))
        with open(os.path.join(out_dir, "result.txt"), "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_partitions():
    for k in [0, 1, 5, 12345, 950114]:
        for world in [1, 2, 3, 8]:
            parts = [multi.shard_range(k, r, world) for r in range(world)]
            assert sum(c for _, c in parts) == k
            assert parts[0][0] == 0
            for (f0, c0), (f1, _) in zip(parts, parts[1:]):
                assert f0 + c0 == f1


def test_sharded_counts_sum_exactly_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert (tmp_path / "result.txt").read_text() == "ok"


def test_oracle_shards_sum_without_collective():
    import graphgen
    import oracle
    src, dst = graphgen.kronecker_host(9)
    off, adj = oracle.csr(src, dst, 512)
    k = 7777
    total = None
    for r in range(3):
        first, cnt = multi.shard_range(k, r, 3)
        p = oracle.sample(off, adj, 2, 2, 5, cnt, cnt, first=first)
        blk = multi.counter_block(p["counts"], int(p["glob"][0]), int(p["glob"][1]), p["stats"]).view(np.uint64)
        total = blk if total is None else total + blk
    full = oracle.sample(off, adj, 2, 2, 5, k, k)
    ref = multi.counter_block(full["counts"], int(full["glob"][0]), int(full["glob"][1]), full["stats"])
    assert np.array_equal(total, ref.view(np.uint64))
