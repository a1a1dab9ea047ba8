"""Benchmark of the wedge-sampling hot path on GB300.

One step = the whole path on one synthetic graph: edge list (resident in HBM)
-> CSR with degrees (expand, radix sort, dedup, offset scan) -> degree bins
and wedge prefix -> per-bin and global wedge sampling with closure checks and
tallies -> FP64 estimates. Workload: Graph500 Kronecker (R-MAT 0.57/0.19/0.19/
0.05), scale 28, edge factor 16 (4,294,967,296 generated edges, ids permuted),
bins 2^i <= d < 2^(i+1), 950,114 samples per nonempty bin and globally
(eps = 0.002, delta = 0.001), Philox seed 7.

Prints one JSON line. `value` is seconds per million undirected edges of the
whole step (lower is better); `gwedges_checked_per_s` is the sampling stage
alone. `e2e` runs the same step through the C ABI from pinned host buffers,
host-to-device copies inside the timed region. `batched` compares 512 plain
single-graph sampling calls with one autotuned persistent launch over the
same 512 requests (Kronecker and Chung-Lu graphs, per-bin budgets 1e3-1e6). `--impl reference` times the
CPU oracle on the host cores on a bounded sample of the workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gwedges checked/s and s per M edges at Kronecker scale 28; batched vs plain"
K_SAMPLES = 950114  # eps = 0.002, delta = 0.001 (Thm 3.1 bound 950,113 rounded as quoted)
SEED = 7
TAU, OMEGA = 1, 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=28)
    ap.add_argument("--edgefactor", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-rounding", action="store_true",
                    help="skip the per-bin variant legs (Phase 2a rounding, sorted closure)")
    ap.add_argument("--tri-k", type=int, default=5_000_000,
                    help="samples of the triangle-statistics leg (Sec. 5.7 single-bin run; 0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests per rate for the serving sweep (the full sweep uses 10000; 0 skips it)")
    ap.add_argument("--serve-rates", default="300,3000", help="arrival rates per second (full sweep: "
                                                             "100,300,1000,3000,5000)")
    ap.add_argument("--serve-batch-samples", type=int, default=4_000_000,
                    help="serving: samples a batch may take (a larger request goes alone)")
    ap.add_argument("--serve-filling-samples", type=int, default=4_000_000,
                    help="serving: a batch this large fills the GPU; two such batches do not run together")
    ap.add_argument("--serve-queue-samples", type=int, default=500_000_000,
                    help="serving: queued samples beyond which a submit is refused (WEDGE_EBUSY)")
    ap.add_argument("--probe-gb", type=int, default=32,
                    help="buffer of the random-read roofline probe, GB (much larger than L2)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched leg: the configuration the autotuner picks on this mix (thread mapping, 512 "
                         "threads, 4096-sample tiles) instead of tuning (for profiling the persistent launch)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# --------------------------------------------------------------------------
# Clock sampling during the timed region
# --------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# Reference arm: the CPU oracle on the host cores
# --------------------------------------------------------------------------

def oracle_step(scale: int, edgefactor: int, k: int):
    """One full oracle pass (CSR, bins, sampling, estimates) on a Kronecker
    graph of the given scale; returns (seconds, undirected edges, samples)."""
    import graphgen
    import oracle
    from oracle.estimate import estimate
    src, dst = graphgen.kronecker_host(scale, n_edges=edgefactor << scale, seed=1)
    t0 = time.perf_counter()
    off, adj = oracle.csr(src, dst, 1 << scale)
    bb = oracle.bins(off, TAU, OMEGA)
    r = oracle.sample(off, adj, TAU, OMEGA, SEED, k, k)
    estimate(bb["p_b"], r["counts"], r["glob"], 0.001)
    dt = time.perf_counter() - t0
    n_samples = int(r["counts"][:, 0].sum()) + int(r["glob"][0])
    return dt, adj.shape[0] // 2, n_samples


def modelled_sampler_sectors(wedge, torch, g, b, k_bin, k_glob, hot_levels=20):
    """The random-access model of one sample (32-byte sectors, one per
    random access): the centre search over the stream's prefix W (uint64,
    4 per sector, ceil(log2(len/4)) levels) + L[j] + off[v0] + adj[i], adj[j]
    + off[v1], off[v2] + the closure search in the smaller row (int32, 8 per
    sector, ceil(log2(d_lo/8)) levels + 1); the top `hot_levels` levels of
    either search stay in L2. Centre searches use each stream's actual length
    (bin sizes); the closure term uses the degrees of a recorded draw of the
    global stream. Returns sectors per sample over the step's streams."""
    import numpy as np
    bi = b.info()
    k = min(k_glob, 1 << 20)
    rec = torch.zeros(k * 8, dtype=torch.int32, device="cuda")
    wedge.sample(g, b, seed=SEED + 1, k_global=k, flags=wedge.FLAG_NO_BINS, records=rec)
    r = rec.cpu().numpy().reshape(-1, 8).astype(np.int64)
    d1, d2 = r[:, 5], r[:, 6]
    dlo = np.minimum(d1, d2)
    closure = np.maximum(0, np.ceil(np.log2(np.maximum(dlo, 1) / 8.0)) - hot_levels) + 1
    per_sample = 6.0 + float(closure.mean())

    def centre(length):
        return max(0.0, math.ceil(math.log2(max(length, 1) / 4.0)) - hot_levels)

    total, count = 0.0, 0
    for bid in range(2, bi.n_bins):
        nb = int(bi.start[bid + 1] - bi.start[bid])
        if int(bi.p_b[bid]) > 0 and nb > 0:
            total += k_bin * (centre(nb) + per_sample)
            count += k_bin
    total += k_glob * (centre(int(bi.n_wedge_vertices)) + per_sample)
    count += k_glob
    return total / count


def cpu_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # Bounded sample: the largest scale whose whole run fits a few minutes.
    scale = 20 if args.steps + args.warmup <= 8 else 18
    for _ in range(args.warmup):
        oracle_step(scale, args.edgefactor, K_SAMPLES)
    times, m, ns = [], 0, 0
    for _ in range(args.steps):
        dt, m, ns = oracle_step(scale, args.edgefactor, K_SAMPLES)
        times.append(dt)
    t = sum(times) / len(times)
    value = t / (m / 1e6)
    sample = (f"Kronecker scale {scale} (edge factor {args.edgefactor}), full oracle pass: CSR, bins, "
              f"{K_SAMPLES} samples per nonempty bin and globally, estimates")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/Medge", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"kronecker-s{scale}-ef{args.edgefactor} (bounded sample of kronecker-s28)",
                       "scale": scale, "k_per_bin": K_SAMPLES, "k_global": K_SAMPLES, "tau": TAU, "omega": OMEGA},
            "gwedges_checked_per_s": ns / t / 1e9,
            "cpu_baseline": {"value": value, "unit": "s/Medge", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "s/Medge", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# Our arm
# --------------------------------------------------------------------------

KERNEL_SOURCES = {
    # the sources a kernel's counters depend on; ncu figures are void once these change
    "sort_onesweep_pass": ["sort.cu", "device.cuh"],
    "sample_closure": ["sample.cu", "sample_device.cuh", "device.cuh"],
    "dedup_rows": ["graph.cu", "device.cuh"],
    "expand_edges": ["graph.cu"],
    "edge_histograms": ["graph.cu"],
    "probe_random_read": ["probe.cu"],
    "merge_runs": ["merge.cu"],
    "batch_sample": ["batch.cu", "sample_device.cuh", "device.cuh"],
}


def host_available_bytes():
    """MemAvailable from /proc/meminfo, or None where it cannot be read."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_1301_5887_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_figures(kernel):
    """Counters of `kernel` from profiles/traffic.json if they were taken on
    the current source, else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        ent = json.load(f).get(kernel)
    if not ent or ent.get("source_hash") != source_hash(kernel):
        return None
    return ent


ALG_BYTES = {
    # algorithmic DRAM bytes per launch, from the sizes of one step.
    # sort_onesweep_pass: the mean over the step's passes of 16 B per key
    # (8 read + 8 written) for the forward passes (one key per generated edge;
    # the first reads the edge's two int32 endpoints) and the transposed ones
    # (one key per unique edge, m = n_adj / 2), except the last transposed pass,
    # which reads 8 B and writes one 4 B adjacency entry per key
    "sort_onesweep_pass": lambda z: z["sort_bytes"] / z["sort_launches"],
    "sort_histogram": lambda z: 8 * z["nkeys"],
    "edge_histograms": lambda z: 8 * z["n_edges"],
    "expand_edges": lambda z: 16 * z["n_edges"],
    "dedup_rows": lambda z: 8 * z["n_edges"] + 4 * z["n_adj"],  # keys in, transposed keys of the unique ones out
    "place_rows": lambda z: 8 * z["n_edges"] + 2 * z["n_adj"],  # sorted keys in again, 4-byte entries out
    "row_offsets": lambda z: 36 * z["n"],
    "scan_degrees": lambda z: 12 * z["n"],
    "bin_count": lambda z: 4 * z["n"],
    "bin_scatter": lambda z: 4 * z["n"] + 12 * z["n2"],
    "scan_bin_wedges": lambda z: 16 * z["n2"],
}


def sort_sizes(n_edges, n_adj, id_bits):
    """Sort passes of one CSR build: ceil(2b/8) over the forward keys, then
    ceil(b/8) over the transposed ones. Returns (mean keys per pass, passes,
    algorithmic bytes of all passes)."""
    pf, pt = (2 * id_bits + 7) // 8, (id_bits + 7) // 8
    m = n_adj // 2
    nbytes = 16 * pf * n_edges + 16 * (pt - 1) * m + 12 * m
    return (pf * n_edges + pt * m) / (pf + pt), pf + pt, nbytes


def build_batched_mix(wedge, graphgen, torch, n_graphs=512, seed=3):
    """The batched workload: half Kronecker graphs with scales drawn
    log-uniformly from 8-22, half Chung-Lu power-law graphs (exponent
    U(2.0, 2.6), mean degree U(8, 64), 2^U{10..22} vertices); per-bin and
    global budgets drawn log-uniformly from [1e3, 1e6]."""
    import numpy as np
    rng = np.random.default_rng(seed)
    stream = torch.cuda.current_stream().cuda_stream
    items, edges = [], 0
    for i in range(n_graphs):
        if i < n_graphs // 2:
            scale = int(round(float(np.exp(rng.uniform(np.log(8), np.log(22))))))
            n, m = 1 << scale, graphgen.kronecker_edges(scale)
            s = torch.empty(m, dtype=torch.int32, device="cuda")
            d = torch.empty(m, dtype=torch.int32, device="cuda")
            graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), m, stream, seed=10_000 + i)
            kind = f"kronecker-s{scale}"
        else:
            n = 1 << int(rng.integers(10, 23))
            gamma, dbar = float(rng.uniform(2.0, 2.6)), float(rng.uniform(8, 64))
            prefix, m = graphgen.chunglu_weights(n, gamma, dbar)
            pd = torch.as_tensor(prefix.view(np.int64)).cuda()
            s = torch.empty(m, dtype=torch.int32, device="cuda")
            d = torch.empty(m, dtype=torch.int32, device="cuda")
            graphgen.chunglu_device(pd.data_ptr(), n, s.data_ptr(), d.data_ptr(), m, 20_000 + i, stream_ptr=stream)
            kind = f"chunglu-n{n}"
        g = wedge.graph_build(s, d, n)
        del s, d
        b = wedge.bin(g, tau=TAU, omega=OMEGA)
        nb = b.info().n_bins
        k_bin = np.exp(rng.uniform(np.log(1e3), np.log(1e6), nb)).astype(np.uint64)
        k_glob = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        items.append({"graph": g, "bins": b, "seed": 30_000 + i, "k_bin": k_bin, "k_global": k_glob, "kind": kind})
        edges += m
    return items, edges


def bench_batched(wedge, graphgen, torch, probe_rate=None, probe_spa=None, autotune=True, probe_l2=None):
    """512 plain wedge_sample calls vs one autotuned persistent launch; the
    persistent launch's random-access roofline fraction where DRAM sector
    counters of that kernel on this mix exist for the current source."""
    import numpy as np
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    items, edges = build_batched_mix(wedge, graphgen, torch)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    reqs = wedge.Requests(items)
    t0 = time.perf_counter()
    if autotune:
        cfg = wedge.autotune(reqs)
    else:
        cfg = wedge.LaunchConfig(wedge.MAP_THREAD, wedge.MAP_THREAD, wedge.MAP_THREAD, 512, 4096, 0)
    tune_s = time.perf_counter() - t0

    def plain():
        return [wedge.sample(it["graph"], it["bins"], seed=it["seed"], k_global=it["k_global"], k_bin=it["k_bin"])
                for it in items]

    plain()  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = plain()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0

    wedge.sample_batch(reqs, cfg=cfg)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = wedge.sample_batch(reqs, cfg=cfg)
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t0

    batch = wedge.Batch(reqs, cfg=cfg)
    batch.launch()
    batch.results()
    t0 = time.perf_counter()
    batch.launch()
    got2 = batch.results()
    replay_s = time.perf_counter() - t0
    info = batch.info()
    batch.free()

    identical = all(np.array_equal(a.counts_matrix(), b.counts_matrix()) and a.closed_global == b.closed_global
                    and np.array_equal(a.stats, b.stats) for a, b in zip(ref, got)) and \
        all(np.array_equal(a.counts_matrix(), b.counts_matrix()) for a, b in zip(ref, got2))
    samples = sum(int(c.k_b.sum()) + c.k_global for c in ref)
    for it in items:
        it["bins"].free()
        it["graph"].free()
    # Every graph of the mix has at most 2^22 vertices, so in the access model
    # (modelled_sampler_sectors) all search levels stay in L2: 7 random
    # accesses per sample (6 gathers + the last closure probe), and most of
    # the mix's working set is L2-resident (ncu: a few DRAM sectors per
    # sample). The ceiling is then the rate of random reads that hit L2.
    s_mix = 7.0
    roof = {"bound": "random-access (L2-resident working set)", "kernel": "batch_sample",
            "modelled_accesses_per_sample": s_mix, "unit": "G accesses/s",
            "achieved": s_mix * samples / batch_s / 1e9,
            "peak": probe_l2 / 1e9 if probe_l2 else None,
            "frac": s_mix * samples / batch_s / probe_l2 if probe_l2 else None,
            "peak_source": "wedge_probe_random_read live over a 64 MB buffer (L2-resident), best of 3"}
    ent = ncu_figures("batch_sample")
    if ent and ent.get("samples") == samples and probe_rate and probe_spa:
        spl = ent["dram_sectors_per_sample"]
        roof["dram"] = {"dram_sectors_per_sample": spl, "achieved_gbs": spl * samples / batch_s * 32 / 1e9,
                        "dram_random_peak_gbs": probe_rate * probe_spa * 32 / 1e9,
                        "frac": spl * samples / batch_s / (probe_rate * probe_spa)}
    return {"workload": "512 graphs: 256 Kronecker (scale log-uniform 8-22) + 256 Chung-Lu (exponent 2.0-2.6, "
                        "mean degree 8-64, 2^10-2^22 vertices); per-bin and global budgets log-uniform 1e3-1e6",
            "graphs": len(items), "generated_edges": edges, "samples": samples,
            "plain_calls": len(items), "plain_s": plain_s, "plain_gwedges_per_s": samples / plain_s / 1e9,
            "batched_s": batch_s, "batched_gwedges_per_s": samples / batch_s / 1e9,
            "replay_s": replay_s, "replay_gwedges_per_s": samples / replay_s / 1e9,
            "speedup": plain_s / batch_s, "identical_to_plain": bool(identical),
            "tuned_config": cfg.as_dict(), "autotuned": autotune, "tiles": info["tiles"],
            "persistent_grid": info["grid"], "setup_s": setup_s, "tune_s": tune_s, "roofline": roof}


def bench_serving(wedge, graphgen, torch, rates, n_requests, n_graphs=64, seed=5, upload_frac=0.01,
                  batch_samples=4_000_000, filling_samples=4_000_000, queue_samples=500_000_000):
    """Poisson request stream against a resident pool of Kronecker and
    Chung-Lu graphs (scales 14-24) under a 150 GB HBM budget; per-request eps
    drawn from {0.01, 0.005, 0.002}, delta 0.001; 1% of arrivals upload a new
    edge list. For each rate: p50/p99 latency and Gwedges/s of the
    continuous-batching server, against a plain path that runs the same
    requests one wedge_sample call at a time in arrival order."""
    import threading

    import numpy as np
    rng = np.random.default_rng(seed)
    stream = torch.cuda.current_stream().cuda_stream

    def gen_edges(i):
        if i % 2 == 0:
            scale = int(rng.integers(14, 25))
            n, m = 1 << scale, graphgen.kronecker_edges(scale)
            s = torch.empty(m, dtype=torch.int32, device="cuda")
            d = torch.empty(m, dtype=torch.int32, device="cuda")
            graphgen.kronecker_device(scale, s.data_ptr(), d.data_ptr(), m, stream, seed=40_000 + i)
        else:
            n = 1 << int(rng.integers(14, 25))
            prefix, m = graphgen.chunglu_weights(n, float(rng.uniform(2.0, 2.6)), float(rng.uniform(8, 32)))
            pd = torch.as_tensor(prefix.view(np.int64)).cuda()
            s = torch.empty(m, dtype=torch.int32, device="cuda")
            d = torch.empty(m, dtype=torch.int32, device="cuda")
            graphgen.chunglu_device(pd.data_ptr(), n, s.data_ptr(), d.data_ptr(), m, 50_000 + i, stream_ptr=stream)
        torch.cuda.synchronize()
        return s, d, n

    # Admission: at most ~50 ms of queued work at the GPU's ~10 Gwedges/s;
    # batches capped at 4M samples (~0.5 ms of work); one GPU-filling batch at a time.
    srv = wedge.Server(hbm_budget_bytes=150 * 10**9, slots=2,
                       launch={"block_threads": 512, "samples_per_tile": 4096, "flags": wedge.BATCH_DIRECT},
                       max_batch_samples=batch_samples, max_queued_samples=queue_samples,
                       gpu_filling_samples=filling_samples)
    ids, plain = [], []
    for i in range(n_graphs):
        s, d, n = gen_edges(i)
        ids.append(srv.add_graph(s, d, n))
        g = wedge.graph_build(s, d, n)
        plain.append((g, wedge.bin(g, tau=TAU, omega=OMEGA)))
        del s, d
    torch.cuda.empty_cache()
    eps_set = [0.01, 0.005, 0.002]
    out = []
    for rate in rates:
        gaps = rng.exponential(1.0 / rate, n_requests)
        arrivals = np.cumsum(gaps)
        reqs = [(int(rng.integers(0, len(ids))), int(rng.integers(1, 1 << 40)), float(rng.choice(eps_set)),
                 bool(rng.random() < upload_frac)) for _ in range(n_requests)]
        # the uploads' edge lists, generated before either timed loop: both
        # paths upload the same graphs
        up_edges = {j: gen_edges(1000 + j) for j in range(n_requests) if reqs[j][3]}
        # continuous-batching server
        srv.stats(reset=True)
        tickets = [None] * n_requests
        uploads = []

        def uploader(i):
            s, d, n = up_edges[i]
            try:
                t0 = time.perf_counter()
                srv.add_graph(s, d, n)
                uploads.append(time.perf_counter() - t0)
            except wedge.WedgeError:
                uploads.append(None)

        up_threads = []
        t_start = time.perf_counter()
        for j, (gi, sd, eps, is_upload) in enumerate(reqs):
            delay = t_start + arrivals[j] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            if is_upload:
                th = threading.Thread(target=uploader, args=(j,))
                th.start()
                up_threads.append(th)
            try:
                tickets[j] = srv.submit(ids[gi], sd, eps=eps, delta=0.001)
            except wedge.WedgeError as e:  # admission control: the queue holds ~50 ms of work
                if e.status != wedge.EBUSY:
                    raise
        for t in tickets:
            if t is not None:
                srv.wait(t)
        for th in up_threads:
            th.join()
        st = srv.stats(reset=True)
        # plain per-request path, same arrivals and uploads, one call at a time
        lat = []
        samples = 0
        t_start = time.perf_counter()
        for j, (gi, sd, eps, is_upload) in enumerate(reqs):
            delay = t_start + arrivals[j] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            if is_upload:
                s_, d_, n_ = up_edges[j]
                gu = wedge.graph_build(s_, d_, n_)
                bu = wedge.bin(gu, tau=TAU, omega=OMEGA)
                bu.free()
                gu.free()
                up_edges[j] = None
            g, b = plain[gi]
            c = wedge.sample(g, b, seed=sd, eps=eps, delta=0.001)
            done = time.perf_counter()
            lat.append((done - (t_start + arrivals[j])) * 1e6)
            samples += int(c.k_b.sum()) + c.k_global
        span = time.perf_counter() - t_start
        lat.sort()

        def pct(v, p):
            return v[max(1, int(np.ceil(p * len(v)))) - 1]

        out.append({"rate_per_s": rate, "requests": n_requests,
                    "served": {"rejected": int(st["rejected_requests"]),
                               "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                               "gwedges_per_s": st["samples"] / st["span_s"] / 1e9 if st["span_s"] else None,
                               "requests_per_s": st["completed"] / st["span_s"] if st["span_s"] else None,
                               "mean_batch_requests": st["mean_batch_requests"], "batches": st["batches"]},
                    "plain": {"p50_ms": pct(lat, 0.5) / 1e3, "p99_ms": pct(lat, 0.99) / 1e3,
                              "gwedges_per_s": samples / span / 1e9, "requests_per_s": n_requests / span},
                    "uploads": len(uploads), "uploads_rejected": sum(1 for u in uploads if u is None)})
    res_bytes = srv.stats()["resident_bytes"]
    srv.close()
    for g, b in plain:
        b.free()
        g.free()
    return {"workload": f"{n_graphs} resident graphs (half Kronecker, half Chung-Lu, scales 14-24) under a 150 GB "
                        f"budget; Poisson arrivals; eps in {{0.01, 0.005, 0.002}}, delta 0.001; "
                        f"{upload_frac:.0%} uploads",
            "policy": f"batches in arrival order up to {batch_samples:,} samples; one GPU-filling "
                      f"(>= {filling_samples:,} samples) batch at a time, smaller requests overtake queued large "
                      f"ones; submits refused (WEDGE_EBUSY) past {queue_samples:,} queued samples; latency "
                      f"percentiles over admitted requests",
            "resident_bytes": res_bytes, "rates": out}


def bench_rounding(wedge, graphgen, torch, g, b, iid_sampling_ms, reps=3, var_scale=18, var_seeds=24):
    """Per-bin sampling by per-vertex probabilistic rounding (Alg. Phase 2a/2c)
    against the i.i.d. inverse-CDF streams on the resident graph: time per
    call (kernels from the profiler), and on a smaller graph the spread of the
    per-bin estimates c_b over seeds for both allocations."""
    import numpy as np
    flags = wedge.FLAG_ROUNDING | wedge.FLAG_NO_GLOBAL
    wedge.sample(g, b, seed=SEED, k_per_bin=K_SAMPLES, flags=flags)
    wedge.profile_reset()
    wedge.profile_enable(True)
    for r in range(reps):
        c = wedge.sample(g, b, seed=SEED + r, k_per_bin=K_SAMPLES, flags=flags)
    wedge.profile_enable(False)
    prof = wedge.profile_read()
    names = ("round_alloc", "scan_round_counts", "round_bin_base", "round_draw")
    per = {k: prof[k]["total_ms"] / reps for k in names if k in prof}
    total_ms = sum(per.values())
    samples = int(c.k_b.sum())
    # estimator spread: same k per bin, many seeds, both allocations
    s, d = graphgen.kronecker_host(var_scale, seed=2)
    gs = wedge.graph_build(s, d, 1 << var_scale)
    bs = wedge.bin(gs, tau=TAU, omega=OMEGA)
    kv = 20000
    est = {"iid": [], "rounding": []}
    for seed in range(var_seeds):
        ci = wedge.sample(gs, bs, seed=100 + seed, k_per_bin=kv, flags=wedge.FLAG_NO_GLOBAL)
        cr = wedge.sample(gs, bs, seed=100 + seed, k_per_bin=kv, flags=flags)
        for key, cc in (("iid", ci), ("rounding", cr)):
            kb = cc.k_b.astype(np.float64)
            closed = cc.q[:, 1:].sum(axis=1).astype(np.float64)
            est[key].append(np.where(kb > 0, closed / np.maximum(kb, 1), np.nan))
    spread = {}
    for key in est:
        a = np.array(est[key])
        a = a[:, np.isfinite(a).sum(axis=0) >= 2]  # bins sampled under at least two seeds
        m = np.nanmean(a, axis=0)
        sd = np.nanstd(a, axis=0, ddof=1)
        ok = m > 0
        spread[key] = float(np.nanmedian(sd[ok] / m[ok]))
    bs.free()
    gs.free()
    return {"ms": total_ms, "kernels_ms": per, "samples": samples,
            "gwedges_per_s": samples / (total_ms / 1e3) / 1e9 if total_ms > 0 else None,
            "iid_sampling_ms_same_budget": iid_sampling_ms,
            "median_rel_std_c_b": spread, "spread_workload": f"kronecker-s{var_scale}, k_b = {kv}, {var_seeds} seeds",
            "note": "rounding: allocation + scan + bin bases + draws over the bins' streams (no global stream); "
                    "iid_sampling_ms_same_budget includes the global stream's K samples as well"}


def bench_sorted_closure(wedge, g, b, reps=3):
    """Per-bin sampling with closure checked in sorted order against the inline
    check, same samples (identical counts), at the bench budget and 8x it."""
    import numpy as np
    out = []
    for mult in (1, 8):
        k = K_SAMPLES * mult
        row = {"k_per_bin": k}
        for name, flags in (("inline", wedge.FLAG_NO_GLOBAL),
                            ("sorted", wedge.FLAG_SORTED_CLOSURE | wedge.FLAG_NO_GLOBAL)):
            c = wedge.sample(g, b, seed=SEED, k_per_bin=k, flags=flags)
            wedge.profile_reset()
            wedge.profile_enable(True)
            for r in range(reps):
                c = wedge.sample(g, b, seed=SEED, k_per_bin=k, flags=flags)
            wedge.profile_enable(False)
            prof = wedge.profile_read()
            ms = sum(v["total_ms"] for v in prof.values()) / reps
            row[name] = {"ms": ms, "kernels_ms": {kk: v["total_ms"] / reps for kk, v in prof.items()},
                         "gwedges_per_s": int(c.k_b.sum()) / (ms / 1e3) / 1e9}
            row[name + "_counts"] = c.counts_matrix()
        row["identical"] = bool(np.array_equal(row.pop("inline_counts"), row.pop("sorted_counts")))
        out.append(row)
    return out


def compact_summary(value, ms_step, gwps, roofline, sampling_roofline, e2e, batched, serving):
    """The headline figures in a few hundred bytes (the end of the JSON line)."""
    def r(x, nd=4):
        return round(x, nd) if isinstance(x, float) else x
    out = {"s_per_Medge": value, "ms_per_step": r(ms_step, 2), "gwedges_checked_per_s": r(gwps, 3),
           "sort_pass_frac_of_copy_peak": r(roofline["frac"], 3),
           "sampler_frac_of_random_access_peak": r(sampling_roofline.get("frac"), 3),
           "sampler_modelled_sectors_per_sample": r(sampling_roofline.get("modelled_sectors_per_sample"), 2),
           "e2e_ms_per_step": r(e2e.get("ms_per_step"), 1) if e2e else None,
           "e2e_h2d_link_gbs": r(e2e.get("h2d_link_gbs"), 1) if e2e else None}
    if batched:
        out["batched"] = {"plain_gwps": r(batched["plain_gwedges_per_s"], 3),
                          "batched_gwps": r(batched["batched_gwedges_per_s"], 3),
                          "replay_gwps": r(batched["replay_gwedges_per_s"], 3),
                          "speedup": r(batched["speedup"], 3), "identical_to_plain": batched["identical_to_plain"],
                          "roofline_frac": r(batched.get("roofline", {}).get("frac"), 3)}
    if serving:
        out["serving"] = [{"rate": row["rate_per_s"],
                           "served_p50_ms": r(row["served"]["p50_ms"], 2), "served_p99_ms": r(row["served"]["p99_ms"], 2),
                           "plain_p50_ms": r(row["plain"]["p50_ms"], 2), "plain_p99_ms": r(row["plain"]["p99_ms"], 2),
                           "served_gwps": r(row["served"]["gwedges_per_s"], 3),
                           "plain_gwps": r(row["plain"]["gwedges_per_s"], 3),
                           "rejected": row["served"].get("rejected", 0)}
                          for row in serving["rates"]]
    return out


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    import graphgen
    import paper_1301_5887_gb300 as wedge

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    __graft_entry__.build() if rank == 0 and world == 1 else None
    if world > 1:
        if rank == 0:
            __graft_entry__.build()
        dist.barrier()
    wedge.load()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    scale, ef = args.scale, args.edgefactor
    n = 1 << scale
    n_edges = ef << scale
    src = torch.empty(n_edges, dtype=torch.int32, device="cuda")
    dst = torch.empty(n_edges, dtype=torch.int32, device="cuda")
    graphgen.kronecker_device(scale, src.data_ptr(), dst.data_ptr(), n_edges, stream.cuda_stream, seed=1)
    torch.cuda.synchronize()

    info = {}

    def step(s_in, d_in):
        g = wedge.graph_build(s_in, d_in, n)
        b = wedge.bin(g, tau=TAU, omega=OMEGA)
        c = wedge.sample(g, b, seed=SEED, k_per_bin=K_SAMPLES, k_global=K_SAMPLES)
        est = wedge.estimate(c, 0.001)
        gi, bi = g.info(), b.info()
        info.update(n_adj=gi.n_adj, n2=bi.n_wedge_vertices, n_bins=bi.n_bins,
                    samples=int(c.k_b.sum()) + c.k_global, c_hat=est["c_hat"], c_hat_global=est["c_hat_global"],
                    n_streams=int((c.k_b > 0).sum()) + (1 if c.k_global else 0),
                    counts=(c.q.tobytes(), c.k_b.tobytes(), c.k_global, c.closed_global, gi.n_adj))
        b.free()
        g.free()

    for _ in range(args.warmup):
        step(src, dst)

    # Timed region: device-resident inputs (34 GB at scale 28 >> 129 MB L2).
    clocks = Clocks(dev)
    clocks.start()
    wedge.profile_reset()
    wedge.profile_enable(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(src, dst)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wedge.profile_enable(False)
    ms_total = e0.elapsed_time(e1)
    prof = wedge.profile_read()
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms_total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    m = info["n_adj"] // 2
    value = (ms_step / 1e3) / (world * m / 1e6)
    samp = prof.get("sample_closure", {"total_ms": 0.0, "launches": 0})
    samp_ms = samp["total_ms"] / max(samp["launches"], 1)
    gwps = world * info["samples"] / (samp_ms / 1e3) / 1e9 if samp_ms > 0 else None
    launches = sum(v["launches"] for v in prof.values())

    nkeys, sort_launches, sort_bytes = sort_sizes(n_edges, info["n_adj"], scale)
    sizes = {"nkeys": nkeys, "sort_launches": sort_launches, "sort_bytes": sort_bytes, "n_edges": n_edges,
             "n_adj": info["n_adj"], "n": n, "n2": info["n2"]}
    top = max((k for k in prof if k in ALG_BYTES), key=lambda k: prof[k]["total_ms"])
    peaks, peak_kind = measured_peaks()
    avg_ms = prof[top]["total_ms"] / prof[top]["launches"]
    achieved = ALG_BYTES[top](sizes) / (avg_ms / 1e3) / 1e9
    traffic = None
    ent = ncu_figures(top)
    if ent and ent.get("bytes_per_unit"):  # DRAM read+write bytes per key (or edge), scaled to this launch
        traffic = ent["bytes_per_unit"] * sizes[ent["unit"]]
    roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "alg_bytes_per_launch": ALG_BYTES[top](sizes), "avg_launch_ms": avg_ms}

    kernels = {k: {"launches": v["launches"] // args.steps, "ms_per_step": v["total_ms"] / args.steps,
                   "share": v["total_ms"] / max(ms_total, 1e-9)} for k, v in prof.items()}

    # Sampling-stage roofline: the sampler's DRAM sector rate against the rate
    # random reads can move sectors on this GPU. Random reads are probed live
    # (accesses/s); sectors per sample and per probe access come from ncu
    # counters taken on the current kernel sources (null otherwise).
    # Model of the sampler's random accesses on this graph (sectors per sample).
    g_m = wedge.graph_build(src, dst, n)
    b_m = wedge.bin(g_m, tau=TAU, omega=OMEGA)
    s_alg = modelled_sampler_sectors(wedge, torch, g_m, b_m, K_SAMPLES, K_SAMPLES)
    b_m.free()
    g_m.free()
    wedge.trim()
    probe = wedge.probe_random_read(args.probe_gb << 30, 1 << 30)
    probe_l2 = wedge.probe_random_read(64 << 20, 1 << 30)  # random reads that hit L2
    sent, pent = ncu_figures("sample_closure"), ncu_figures("probe_random_read")
    spa = pent["dram_sectors_per_access"] if pent else None
    rate = info["samples"] / (samp_ms / 1e3) if samp_ms > 0 else None
    # Algorithmic roofline: the model's random accesses per second against the
    # probe's independent random reads per second (one sector each).
    sampling_roofline = {"bound": "random-access", "kernel": "sample_closure", "unit": "G accesses/s",
                         "modelled_sectors_per_sample": s_alg,
                         "achieved": s_alg * rate / 1e9 if rate else None, "peak": probe / 1e9,
                         "frac": s_alg * rate / probe if rate else None,
                         "probe_accesses_per_s": probe, "probe_dram_sectors_per_access": spa,
                         "probe_l2_accesses_per_s": probe_l2,
                         "peak_source": f"wedge_probe_random_read live (2^30 independent 4-byte reads over "
                                        f"{args.probe_gb} GB, best of 3)"}
    if sent and spa:
        # DRAM sectors per sample measured by ncu on a smaller graph of the same
        # family, beside the model's sectors at that size x the DRAM sectors one
        # random access moves
        sampling_roofline["measured"] = {
            "scale": sent.get("scale"), "dram_sectors_per_sample": sent["dram_sectors_per_sample"],
            "modelled_sectors_per_sample_at_that_scale": sent.get("modelled_sectors_per_sample"),
            "modelled_dram_sectors_per_sample_at_that_scale":
                sent["modelled_sectors_per_sample"] * spa if sent.get("modelled_sectors_per_sample") else None}
        if sent.get("scale") == scale:
            sampling_roofline["dram_frac"] = sent["dram_sectors_per_sample"] * rate / (probe * spa) if rate else None

    # e2e: the same step from pinned host buffers through the C ABI, each step
    # timed on its own (the host link is shared with the node's other tenants).
    e2e = None
    e2e_room = args.e2e_steps > 0
    if e2e_room:
        # Every rank on this node pins its own copy of the edge list: where the
        # node's free host memory cannot hold them all, the leg is skipped and
        # the line says why (all ranks take the same decision).
        local_world = int(os.environ.get("LOCAL_WORLD_SIZE", str(world)))
        need = local_world * 8 * n_edges
        avail = host_available_bytes()
        e2e_room = avail is None or need <= 0.8 * avail
        if world > 1:
            flag = torch.tensor([1 if e2e_room else 0], device="cuda", dtype=torch.int32)
            dist.all_reduce(flag, op=dist.ReduceOp.MIN)
            e2e_room = bool(flag.item())
        if not e2e_room:
            e2e = {"value": None, "unit": "s/Medge", "h2d_bytes_per_step": 8 * n_edges, "d2h_bytes_per_step": None,
                   "skipped": f"host memory: {local_world} rank(s) need {need / 1e9:.1f} GB of pinned edge lists, "
                              f"{(avail or 0) / 1e9:.1f} GB available"}
    if e2e_room:
        hsrc = torch.empty(n_edges, dtype=torch.int32, pin_memory=True)
        hdst = torch.empty(n_edges, dtype=torch.int32, pin_memory=True)
        hsrc.copy_(src)
        hdst.copy_(dst)
        torch.cuda.synchronize()
        # The host link's rate right now (its share of the node's host memory
        # bandwidth varies with the other tenants): a plain copy of the same
        # pinned inputs back over the device arrays, which hold the same values.
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        src.copy_(hsrc, non_blocking=True)
        dst.copy_(hdst, non_blocking=True)
        l1.record(stream)
        torch.cuda.synchronize()
        link_gbs = 8 * n_edges / (l0.elapsed_time(l1) / 1e3) / 1e9
        device_counts = info["counts"]
        step(hsrc, hdst)  # warm the host-input path
        torch.cuda.synchronize()
        # the grouped host path must give the device path's graph and samples
        same_as_device = info["counts"] == device_counts
        times = []
        for _ in range(args.e2e_steps):
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            step(hsrc, hdst)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = sum(times) / len(times)
        if world > 1:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        d2h = 8 + 16 + 2 * 8 * info["n_bins"] + 4 + 8 * (4 * info["n_streams"] + 34 * 34)
        # One more step with the library's per-launch CUDA events on: device
        # time per kernel, and the rest of the wall time (the main stream
        # waiting for host copies, host work between calls).
        wedge.profile_reset()
        wedge.profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(hsrc, hdst)
        torch.cuda.synchronize()
        prof_wall = (time.perf_counter() - t0) * 1e3
        wedge.profile_enable(False)
        eprof = wedge.profile_read()
        kernel_ms = sum(v["total_ms"] for k, v in eprof.items() if k != "h2d_copy")
        e2e = {"value": dt / (world * m / 1e6), "unit": "s/Medge", "h2d_bytes_per_step": 8 * n_edges,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3, "step_ms": [x * 1e3 for x in times],
               "h2d_link_gbs": link_gbs, "h2d_ms_at_link_rate": 8 * n_edges / link_gbs / 1e6,
               "counts_identical_to_device_input": same_as_device,
               "breakdown": {"profiled_step_ms": prof_wall, "kernel_ms": kernel_ms,
                             "not_in_kernels_ms": prof_wall - kernel_ms,
                             "timeline": "per name: [device ms summed over launches, launches, first start, last "
                                         "end], ms after timing was switched on at the step's start",
                             "kernels": {k: [round(v["total_ms"], 2), v["launches"], round(v["first_start_ms"], 2),
                                             round(v["last_end_ms"], 2)]
                                         for k, v in sorted(eprof.items(), key=lambda kv: kv[1]["first_start_ms"])}}}
        del hsrc, hdst

    # Triangle statistics (Sec. 5.7): k global-stream samples, closed ones
    # summarised per BinId(d_min); the call synchronises, so host time is device time.
    tri = None
    rounding = None
    sorted_cl = None
    if args.tri_k > 0 or not args.no_rounding:
        g = wedge.graph_build(src, dst, n)
        b = wedge.bin(g, tau=TAU, omega=OMEGA)
    if not args.no_rounding:
        rounding = bench_rounding(wedge, graphgen, torch, g, b, samp_ms)
        sorted_cl = bench_sorted_closure(wedge, g, b)
    if args.tri_k > 0:
        wedge.triangle_stats(g, b, SEED, args.tri_k)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = wedge.triangle_stats(g, b, SEED, args.tri_k)
            times.append(time.perf_counter() - t0)
        med = sorted(times)[1]
        groups = {int(i): {f: int(r["box"][i, j]) for j, f in enumerate(wedge.BOX_FIELDS)}
                  for i in range(r["box"].shape[0]) if r["box"][i, 0]}
        tri = {"k": args.tri_k, "closed": r["closed"], "ms": med * 1e3, "samples_per_s": args.tri_k / med,
               "ratio_q": [float(x) for x in r["ratio_q"]], "box_by_dmin_bin": groups,
               "note": "median of 3 calls of wedge_triangle_stats on the resident graph (sampling with records, "
                       "key compaction, two radix sorts, box plots)"}
    if args.tri_k > 0 or not args.no_rounding:
        b.free()
        g.free()
        wedge.trim()


    del src, dst
    torch.cuda.empty_cache()

    serving = None
    if args.serve_requests > 0:
        wedge.trim()
        torch.cuda.empty_cache()
        serving = bench_serving(wedge, graphgen, torch, [float(r) for r in args.serve_rates.split(",")],
                                args.serve_requests, batch_samples=args.serve_batch_samples,
                                filling_samples=args.serve_filling_samples, queue_samples=args.serve_queue_samples)
        wedge.trim()

    batched = None
    if not args.no_batched:
        wedge.trim()
        torch.cuda.empty_cache()
        batched = bench_batched(wedge, graphgen, torch, probe_rate=probe, probe_spa=spa,
                                autotune=not args.no_autotune, probe_l2=probe_l2)
        wedge.trim()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, mm, ns = oracle_step(20, ef, K_SAMPLES)
        cpu = {"value": dt / (mm / 1e6), "unit": "s/Medge", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"Kronecker scale 20 (edge factor {ef}, {mm} undirected edges), full oracle pass with "
                         f"{K_SAMPLES} samples per nonempty bin and globally; same metric",
               "seconds": dt, "gwedges_checked_per_s": ns / dt / 1e9}

    if rank == 0:
        # Bulky detail first; the compact figures the step is judged by come
        # last, so that a reader of the line's tail sees them.
        line = {"metric": METRIC, "value": value, "unit": "s/Medge", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": f"kronecker-s{scale}-ef{ef}", "scale": scale, "edgefactor": ef,
                           "n_vertices": n, "generated_edges": n_edges, "undirected_edges": m, "tau": TAU,
                           "omega": OMEGA, "k_per_bin": K_SAMPLES, "k_global": K_SAMPLES, "seed": SEED,
                           "bins": info["n_bins"], "samples_per_step": info["samples"],
                           "l2": f"inputs {8 * n_edges / 1e9:.1f} GB > 129 MB L2, no flush needed",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "kernels": kernels, "triangle_stats": tri, "rounding": rounding, "sorted_closure": sorted_cl,
                "batched": batched, "serving": serving,
                "estimates": {"c_hat": info["c_hat"], "c_hat_global": info["c_hat_global"]},
                "gwedges_checked_per_s": gwps, "sampling_ms": samp_ms,
                "s_per_M_generated_edges": {"device": (ms_step / 1e3) / (world * n_edges / 1e6),
                                            "e2e": (e2e["ms_per_step"] / 1e3) / (world * n_edges / 1e6)
                                            if e2e and e2e.get("ms_per_step") else None},
                "sampling_roofline": sampling_roofline, "cpu_baseline": cpu, "e2e": e2e,
                "roofline": roofline, "gpu_launches": launches // 1, "clocks": clk,
                "summary": compact_summary(value, ms_step, gwps, roofline, sampling_roofline, e2e, batched,
                                           serving)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
