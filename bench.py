#!/usr/bin/env python
"""Benchmark of the multi-scale LFK community-growth hot path on one GB300.

Workload (one step, the default): the 1,000,000-node three-level LFR-style
hierarchical graph (power-law degrees tau = 2.5, mean 30, max 300; micro
community sizes 20..1000, tau = 1.5, grouped 2-6 per level; mixing 0.3 / 0.2 /
0.1; FP32 edge weights uniform in [0.5, 2]), 32 log-spaced scales in
[0.5, 1], every node a seed: graph checks and exact weights, growth of all
32,000,000 (scale, seed) units in one persistent run, dedup per scale, NMI
between successive scales.

  value      seed expansions (units) per second, graph already resident in HBM
  e2e        the same through the C ABI from pinned host buffers, with the
             host->device copy of the graph and the device->host read of every
             scale's communities and the stability inside the timed region
  roofline   growth kernels: algorithmic bytes (4 B per CSR entry scanned, plus
             8 B for the exact weight on a weighted graph, + 16 B per row
             visited) / growth time, against the measured HBM copy bandwidth

--impl reference times the CPU oracle (the reference arm) on a
bounded sample of the same workload.  Under torchrun every rank runs its own
replica of the workload (weak scaling, no collective on the data path).

Other workloads (--workload): lfr-100k (the 100,000-node two-level graph, 20
scales), uneven-batch (256 graphs of log-uniform size as one disjoint union,
16 scales), serve (query server on four 2M-node graphs, Poisson arrivals at
fractions of saturation, p50/p99 latency), full (the paper's whole Alg. 2 on
the 100k-node graph) and accuracy (scale ranges where planted levels are
found, in the shape of the paper's Table 1).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SCALES = 20  # the full method's workload (lfr-100k)
WORKLOAD = ("lfr-100k: 100,000-node LFR-style hierarchical graph (degrees power-law 2.5, mean 20, max 200; "
            "community sizes 20-1000 power-law 1.5; 2 levels, mixing 0.3/0.1; unweighted, seed 1), "
            "20 log-spaced scales in [0.5,1], every node a seed")
GROW_SOURCES = ["paper_1301_0955_gb300/csrc/grow.cu", "paper_1301_0955_gb300/csrc/exact.cuh",
                "paper_1301_0955_gb300/csrc/grow.cuh"]
# DRAM traffic of the growth kernel per workload (ncu capture, see profiles/)
PROFILE_FILES = {"lfr-100k": os.path.join(ROOT, "profiles", "grow_kernel_lfr100k_traffic.json"),
                 "lfr-1m-weighted": os.path.join(ROOT, "profiles", "grow_kernel_lfr1m_weighted_traffic.json")}
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--seeds", type=int, default=0, help="profiling: a seeded sample of this many seeds")
    p.add_argument("--scales", type=int, default=0, help="profiling: fewer scales (0: the workload's)")
    p.add_argument("--flush-mib", type=int, default=1024, help="L2 flush buffer written between steps")
    p.add_argument("--plain-steps", type=int, default=1,
                   help="steps of the plain one-launch-per-scale form timed for comparison (0: skip)")
    p.add_argument("--workload", default="lfr-1m-weighted",
                   choices=["lfr-1m-weighted", "lfr-100k", "uneven-batch", "serve", "full", "accuracy"])
    p.add_argument("--acc-scales", type=int, default=40, help="accuracy: scales in [0.3, 1]")
    p.add_argument("--full-rule", type=int, default=1, help="full: seed rule 1 or 2")
    p.add_argument("--serve-queries", type=int, default=10000, help="serve: queries per load level")
    p.add_argument("--serve-calibration", type=int, default=1000, help="serve: queries of the saturation run")
    p.add_argument("--serve-loads", type=float, nargs="*", default=[0.5, 0.8, 0.95])
    p.add_argument("--serve-workers", type=int, default=4)
    p.add_argument("--serve-batch-units", type=int, default=65536)
    p.add_argument("--serve-node-scale", type=float, default=1.0, help="serve: node count factor")
    p.add_argument("--batch-graphs", type=int, default=256, help="uneven-batch: number of graphs")
    p.add_argument("--batch-node-scale", type=float, default=1.0, help="uneven-batch: node count factor")
    p.add_argument("--batch-scales", type=int, default=16, help="uneven-batch: scales")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value, world):
    """Largest value over the ranks (the whole-job time is the slowest rank's)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, world, max_total_ms):
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank * steps / (max_total_ms / 1e3)


def require_ok(rc, what):
    """A timed step whose call did not return MSCD_OK (0) is not a measurement."""
    if rc != 0:
        raise RuntimeError("%s returned status %d" % (what, rc))


def source_hash():
    h = hashlib.sha256()
    for f in GROW_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        # nvidia-smi samples of the timed region (BENCH_CLOCKS_CSV keeps them)
        self.path = os.environ.get("BENCH_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + CLOCK_QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r["util"] > 0] or rows
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("pcap", "sw_power_cap")):
            if any(r[key].lower().startswith("active") for r in load):
                reasons.append(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load)}


def oracle_units(G, alphas, seeds, threads):
    """One oracle pass (growth + dedup per scale) over `seeds` at every scale;
    returns (units, seconds, edges scanned)."""
    import oracle

    m = len(seeds)
    t0 = time.perf_counter()
    rc, ptr, nodes, f, st = oracle.run(G, alphas, seeds, threads=threads)
    for s in range(len(alphas)):
        lo, hi = s * m, (s + 1) * m
        oracle.dedup(ptr[lo:hi + 1] - ptr[lo], nodes[ptr[lo]:ptr[hi]])
    return m * len(alphas), time.perf_counter() - t0, float(st[:, 0].sum())


def oracle_sample(g, alphas, seconds, threads):
    """Time the oracle (growth + dedup per scale) on a seeded sample of seeds
    at every scale, sized to about `seconds` of CPU time."""
    import oracle

    G = oracle.Graph(g.n, g.row_ptr, g.col, g.w)
    rng = np.random.default_rng(12345)
    m = 8
    while True:
        seeds = np.sort(rng.choice(g.n, m, replace=False)).astype(np.int32)
        units, dt, edges = oracle_units(G, alphas, seeds, threads)
        if dt >= seconds * 0.5 or m >= g.n:
            break
        m = int(min(g.n, max(2 * m, m * seconds / max(dt, 1e-3) * 0.9)))
    return {"value": units / dt, "unit": "units/s", "cores": threads, "kind": "oracle",
            "sample": "%d seeds (seeded) x %d scales = %d units of the same workload, oracle growth + dedup on "
                      "%d host threads, %.1f s" % (m, len(alphas), units, threads, dt),
            "edges_scanned_per_s": edges / dt}


def oracle_sample_batch(graphs, alphas, seconds, threads):
    """The same over the batch: seeded parts in turn, a seeded tenth of each
    part's nodes (at least 8) as seeds, until about `seconds` have passed."""
    import oracle

    rng = np.random.default_rng(12345)
    order = rng.permutation(len(graphs))
    units = 0
    dt = 0.0
    edges = 0.0
    parts = 0
    for p in order:
        g = graphs[p]
        G = oracle.Graph(g.n, g.row_ptr, g.col, g.w)
        m = min(g.n, max(8, g.n // 10))
        seeds = np.sort(rng.choice(g.n, m, replace=False)).astype(np.int32)
        u, t, e = oracle_units(G, alphas, seeds, threads)
        units += u
        dt += t
        edges += e
        parts += 1
        if dt >= seconds:
            break
    return {"value": units / dt, "unit": "units/s", "cores": threads, "kind": "oracle",
            "sample": "%d seeded parts of the batch, a seeded tenth of each part's nodes as seeds x %d scales = "
                      "%d units, oracle growth + dedup on %d host threads, %.1f s" % (parts, len(alphas), units,
                                                                                      threads, dt),
            "edges_scanned_per_s": edges / dt}


# ---------------------------------------------------------------- workloads

class SingleGraph:
    """One resident graph, every scale, every node a seed (or a seeded sample
    of seeds when profiling)."""

    name = ""
    graph_index = 0
    n_scales_full = 0
    description = ""

    def __init__(self, args, scales):
        from paper_1301_0955_gb300 import synth

        self.g = synth.config_graph(self.graph_index)
        self.n_scales = args.scales or self.n_scales_full
        self.alphas = scales(0.5, 1.0, self.n_scales)
        self.seeds_h = None
        if args.seeds:
            self.seeds_h = np.sort(np.random.default_rng(0).choice(self.g.n, args.seeds,
                                                                   replace=False)).astype(np.int32)
        n_seeds = self.g.n if self.seeds_h is None else len(self.seeds_h)
        self.units = self.n_scales * n_seeds
        self.full = self.seeds_h is None and self.n_scales == self.n_scales_full
        self.bytes_per_entry = 4 + (8 if self.g.w is not None else 0)

    def config(self):
        g = self.g
        return {"workload": self.description if self.full else
                "profiling subset: %d seeds x %d scales of the %s workload"
                % (self.units // self.n_scales, self.n_scales, self.name),
                "n_nodes": g.n, "nnz": g.nnz, "weighted": g.w is not None, "scales": self.n_scales,
                "seeds": self.units // self.n_scales}

    def to_device(self, torch, dev):
        g = self.g
        self.rp_d = torch.from_numpy(g.row_ptr).to(dev)
        self.col_d = torch.from_numpy(g.col).to(dev)
        self.w_d = None if g.w is None else torch.from_numpy(g.w).to(dev)
        self.alphas_d = torch.from_numpy(self.alphas).to(dev)
        self.seeds_d = None if self.seeds_h is None else torch.from_numpy(self.seeds_h).to(dev)
        self.rp_h = torch.from_numpy(g.row_ptr).pin_memory().numpy()
        self.col_h = torch.from_numpy(g.col).pin_memory().numpy()
        self.w_h = None if g.w is None else torch.from_numpy(g.w).pin_memory().numpy()
        self.h2d_bytes = int(g.row_ptr.nbytes + g.col.nbytes + (0 if g.w is None else g.w.nbytes)
                             + self.alphas.nbytes + (0 if self.seeds_h is None else self.seeds_h.nbytes))

    def step_resident(self, ctx, stream):
        gid = ctx.load_csr(self.g.n, self.rp_d, self.col_d, self.w_d)
        rc = ctx.run(gid, self.alphas_d, self.seeds_d, stream=stream)
        require_ok(rc, "mscd_run")
        ctx.free_graph(gid)

    def step_e2e(self, ctx):
        gid = ctx.load_csr(self.g.n, self.rp_h, self.col_h, self.w_h)
        rc = ctx.run(gid, self.alphas, self.seeds_h)
        require_ok(rc, "mscd_run")
        nb = read_results(ctx, self.n_scales, 1)
        ctx.free_graph(gid)
        return nb

    step_plain = step_resident

    def cpu_baseline(self, seconds, threads):
        return oracle_sample(self.g, self.alphas, seconds, threads)


class Lfr100k(SingleGraph):
    """The 100,000-node LFR-style graph, 20 scales, every node a seed."""

    name = "lfr-100k"
    graph_index = 1
    n_scales_full = 20
    description = ("lfr-100k: 100,000-node LFR-style hierarchical graph (degrees power-law 2.5, mean 20, max 200; "
                   "community sizes 20-1000 power-law 1.5; 2 levels, mixing 0.3/0.1; unweighted, seed 1), "
                   "20 log-spaced scales in [0.5,1], every node a seed")


class Lfr1mWeighted(SingleGraph):
    """The 1,000,000-node three-level LFR-style graph with FP32 weights, 32
    scales, every node a seed: 32,000,000 units in one run."""

    name = "lfr-1m-weighted"
    graph_index = 2
    n_scales_full = 32
    description = ("lfr-1m-weighted: 1,000,000-node three-level LFR-style hierarchical graph (degrees power-law "
                   "2.5, mean 30, max 300; micro community sizes 20-1000 power-law 1.5, grouped 2-6 per level; "
                   "mixing 0.3/0.2/0.1; FP32 edge weights uniform in [0.5, 2], seed 2), 32 log-spaced scales in "
                   "[0.5,1], every node a seed, all 32M (scale, seed) units in one persistent run")


class UnevenBatch:
    """Many independent graphs of uneven size batched as one disjoint union:
    every seed of every graph at every scale in the same persistent launches."""

    name = "uneven-batch"

    def __init__(self, args, scales):
        import multiprocessing as mp

        from paper_1301_0955_gb300 import synth

        specs = synth.uneven_batch_specs(args.batch_graphs, seed=4, scale_nodes=args.batch_node_scale)
        # generated on the host cores before any GPU call (spawned workers)
        with mp.get_context("spawn").Pool(min(len(specs), os.cpu_count() or 1)) as pool:
            self.graphs = pool.map(synth.graph_from_spec, specs, chunksize=1)
        self.n_scales = args.batch_scales
        self.alphas = scales(0.5, 1.0, self.n_scales)
        self.bytes_per_entry = 4
        self.n_total = sum(g.n for g in self.graphs)
        self.units = self.n_scales * self.n_total
        self.node_scale = args.batch_node_scale

    def config(self):
        ns = [g.n for g in self.graphs]
        return {"workload": "uneven-batch: %d independent two-level LFR-style graphs, node counts log-uniform in "
                            "[1000, 200000] x %g, mean degree 10-40, mixing 0.2-0.4, unweighted, %d log-spaced "
                            "scales in [0.5,1], every node a seed, batched as one disjoint union"
                            % (len(ns), self.node_scale, self.n_scales),
                "graphs": len(ns), "n_nodes": self.n_total, "nnz": sum(g.nnz for g in self.graphs),
                "largest_graph": max(ns), "smallest_graph": min(ns), "scales": self.n_scales,
                "seeds": self.n_total}

    def to_device(self, torch, dev):
        self.dev_parts = [(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev))
                          for g in self.graphs]
        self.alphas_d = torch.from_numpy(self.alphas).to(dev)
        self.host_parts = [(torch.from_numpy(g.row_ptr).pin_memory().numpy(),
                            torch.from_numpy(g.col).pin_memory().numpy()) for g in self.graphs]
        self.h2d_bytes = int(sum(g.row_ptr.nbytes + g.col.nbytes for g in self.graphs) + self.alphas.nbytes)

    def _run(self, ctx, parts, alphas, stream=None):
        gids = [ctx.load_csr(g.n, rp, col) for g, (rp, col) in zip(self.graphs, parts)]
        uid = ctx.graph_union(gids)
        for gid in gids:
            ctx.free_graph(gid)
        rc = ctx.run(uid, alphas, None, stream=stream)
        require_ok(rc, "mscd_run")
        return uid

    def step_resident(self, ctx, stream):
        ctx.free_graph(self._run(ctx, self.dev_parts, self.alphas_d, stream))

    def step_e2e(self, ctx):
        uid = self._run(ctx, self.host_parts, self.alphas)
        nb = read_results(ctx, self.n_scales, len(self.graphs))
        ctx.free_graph(uid)
        return nb

    def step_plain(self, ctx, stream):
        """The plain form: graph after graph, one launch per scale and class."""
        for g, (rp, col) in zip(self.graphs, self.dev_parts):
            gid = ctx.load_csr(g.n, rp, col)
            rc = ctx.run(gid, self.alphas_d, None, stream=stream)
            require_ok(rc, "mscd_run")
            ctx.free_graph(gid)

    def cpu_baseline(self, seconds, threads):
        return oracle_sample_batch(self.graphs, self.alphas, seconds, threads)


WORKLOADS = {"lfr-1m-weighted": Lfr1mWeighted, "lfr-100k": Lfr100k, "uneven-batch": UnevenBatch}


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, np.float64), q)) if len(xs) else None


def serve_phase(ctx, gids, alphas, queries, rate_qps):
    """Offer `queries` (graph, scale index, seeds) at Poisson arrivals of
    `rate_qps` (None: all at once), collect every result; returns latencies
    (submit to done, ms), wall seconds and units."""
    rng = np.random.default_rng(99)
    n = len(queries)
    arrivals = np.zeros(n) if rate_qps is None else np.cumsum(rng.exponential(1.0 / rate_qps, n))
    out = {}
    lat = []
    queued = []
    t0 = time.perf_counter()
    i = 0
    while len(lat) < n:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            g, s, seeds = queries[i]
            out[ctx.submit(gids[g], seeds, alphas[s])] = len(seeds)
            i += 1
        done = [q for q in list(out) if ctx.poll(q) == 2]
        for q in done:
            ptr, nodes, f, t, rc = ctx.result(q, out.pop(q))
            require_ok(rc, "mscd_query_result")
            lat.append(t[2])
            queued.append(t[0])
        if not done:
            time.sleep(0.0002)
    wall = time.perf_counter() - t0
    units = sum(len(q[2]) for q in queries)
    return {"latency_ms": lat, "queue_ms": queued, "wall_s": wall, "units": units}


def run_full(args):
    """The full method (Alg. 2): seeds by rule 1 in a seeded random order,
    carry-over across the 20 scales of the lfr-100k workload, growth, check
    and merge until nothing changes at each scale."""
    from paper_1301_0955_gb300 import build, mscd, synth

    world, rank, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    L = mscd.load()
    g = synth.config_graph(1)
    alphas = mscd.scales_logspaced(0.5, 1.0, N_SCALES)
    prio = np.random.default_rng(11).permutation(g.n).astype(np.int32)
    ctx = mscd.Context(local)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    stream = torch.cuda.current_stream(dev)

    def step():
        require_ok(ctx.full_run(gid, alphas, prio=prio, seed_rule=args.full_rule), "mscd_full_run")

    for _ in range(args.warmup):
        step()
    times = []
    l0 = L.mscd_launch_count()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            step()
            torch.cuda.synchronize(dev)
            times.append((time.perf_counter() - t0) * 1e3)
    launches = L.mscd_launch_count() - l0
    info = [ctx.full_scale(s) for s in range(N_SCALES)]
    grown = sum(i["grown"] for i in info)
    ms = statistics.mean(times)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        G = oracle.Graph(g.n, g.row_ptr, g.col)
        # a bounded sample: the first scales only, until about cpu_seconds pass
        # a bounded sample: the first k scales, k doubling until one run takes
        # about half the budget
        k, dt = 1, 0.0
        while True:
            t0 = time.perf_counter()
            rc, seeds, out = oracle.full(G, alphas[:k], args.full_rule, prio)
            dt = time.perf_counter() - t0
            if dt >= args.cpu_seconds / 2 or k >= N_SCALES:
                break
            k = min(N_SCALES, 2 * k)
        gpu_k = sum(info[s]["grown"] for s in range(k))
        cpu = {"kind": "oracle", "cores": 1, "sample": "the oracle's full method on the same graph and seeds, "
               "the first %d scales, %.1f s" % (k, dt), "value": gpu_k / max(dt, 1e-9),
               "unit": "growth calls/s", "ms_for_these_scales": dt * 1e3}
    line = {"metric": "full method (Alg. 2) run time", "value": ms, "unit": "ms per run", "higher_is_better": False,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic", "dtype": "int64+f64",
            "config": {"workload": WORKLOAD.replace("every node a seed", "seed rule %d in a seeded random order, "
                                                    "eta 0.5" % args.full_rule)},
            "growth_calls": grown, "growth_calls_per_s": grown / (ms / 1e3),
            "seeds": int(len(ctx.full_seeds())),
            "communities_per_scale": [int(len(i["ptr"]) - 1) for i in info],
            "iterations_per_scale": [i["iterations"] for i in info],
            "merges_per_scale": [i["merges"] for i in info],
            "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    ctx.close()


ACC_SETTINGS = [(0.05, 0.2), (0.05, 0.3), (0.2, 0.4), (0.3, 0.4)]  # (macro mu1, micro mu2), Table 1


def planted_cover(labels):
    order = np.argsort(labels, kind="stable").astype(np.int32)
    counts = np.bincount(labels)
    ptr = np.concatenate([[0], np.cumsum(counts[counts > 0])]).astype(np.int64)
    return ptr, order


def scale_ranges(alphas, vals, thr):
    """Scale intervals (in the list's order) where vals >= thr."""
    out, cur = [], None
    for a, v in zip(alphas, vals):
        if v >= thr:
            cur = [a, a] if cur is None else [cur[0], a]
        elif cur is not None:
            out.append(cur)
            cur = None
    if cur is not None:
        out.append(cur)
    return [[round(min(r), 3), round(max(r), 3)] for r in out]


def run_accuracy(args):
    """The shape of the paper's Table 1: at which scales the macro and micro
    communities of two-level LFR-style graphs (n = 10^4, m ~ 10^5) are found,
    for the four mixing settings, by the full method (seed rules 1 and 2) and
    by the independent growth of every seed with dedup."""
    from paper_1301_0955_gb300 import build, mscd, synth

    world, rank, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    build.build()
    alphas = mscd.scales_logspaced(0.3, 1.0, args.acc_scales)
    ctx = mscd.Context(local)
    rows = []
    t_start = time.perf_counter()
    for i, (mu1, mu2) in enumerate(ACC_SETTINGS):
        g = synth.hierarchical_lfr(10_000, 30, 100, 2.0, 1.0, (10, 50), (mu2, mu1), group_range=(2, 6),
                                   seed=200 + i, name="acc-%d" % i)
        gid = ctx.load_csr(g.n, g.row_ptr, g.col)
        planted = [planted_cover(g.labels[1]), planted_cover(g.labels[0])]  # macro, micro
        prio = np.random.default_rng(300 + i).permutation(g.n).astype(np.int32)
        for method in ("full rule 1", "full rule 2", "every seed + dedup"):
            covers = []
            if method.startswith("full"):
                ctx.full_run(gid, alphas, prio=prio, seed_rule=1 if method.endswith("1") else 2)
                for s in range(len(alphas)):
                    r = ctx.full_scale(s)
                    covers.append((r["ptr"], r["nodes"]))
            else:
                ctx.run(gid, alphas)
                for s in range(len(alphas)):
                    ptr, nodes, f, s2c = ctx.communities(s)
                    covers.append((ptr, nodes))
            res = {"mu1": mu1, "mu2": mu2, "method": method}
            for lvl, name in ((0, "macro"), (1, "micro")):
                nm = [ctx.nmi_covers(g.n, c, planted[lvl]) for c in covers]
                b = int(np.nanargmax(nm))
                res[name] = {"best_nmi": round(float(nm[b]), 4), "at_scale": round(float(alphas[b]), 4),
                             "scales_nmi_ge_0.9": scale_ranges(alphas, nm, 0.9),
                             "scales_nmi_ge_0.5": scale_ranges(alphas, nm, 0.5)}
            rows.append(res)
        ctx.free_graph(gid)
    line = {"metric": "scale ranges where planted macro / micro communities are found (Table 1 shape)",
            "value": None, "unit": "scale intervals", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "4 two-level LFR-style graphs, n=10^4, m ~ 9.5*10^4 (degree power law 2, "
                                   "max 100), micro "
                                   "communities 10-50 nodes grouped 2-6 per macro community, (mu1 macro, mu2 "
                                   "micro) in %s; %d log-spaced scales in [0.3, 1]" % (ACC_SETTINGS, len(alphas))},
            "rows": rows, "seconds": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_serve(args):
    """Serving: resident graphs, a Poisson stream of local-community queries,
    continuous batching; p50/p99 latency at fractions of saturation."""
    import multiprocessing as mp

    from paper_1301_0955_gb300 import build, mscd, synth

    world, rank, local = dist_env()
    specs = synth.serving_specs(scale_nodes=args.serve_node_scale)
    with mp.get_context("spawn").Pool(len(specs)) as pool:
        graphs = pool.map(synth.graph_from_spec, specs, chunksize=1)
    sizes = [g.n for g in graphs]
    alphas = None
    import torch

    torch.cuda.set_device(local)
    build.build()
    L = mscd.load()
    alphas = mscd.scales_logspaced(0.5, 1.0, 16)
    ctx = mscd.Context(local)
    gids = [ctx.load_csr(g.n, g.row_ptr, g.col) for g in graphs]
    ctx.serve_start(workers=args.serve_workers, max_batch_units=args.serve_batch_units)
    try:
        # warm-up, then saturation: everything offered at once
        serve_phase(ctx, gids, alphas, synth.serving_queries(50, sizes, seed=6), None)
        sat_q = synth.serving_queries(args.serve_calibration, sizes, seed=8)
        l0 = L.mscd_launch_count()
        sat = serve_phase(ctx, gids, alphas, sat_q, None)
        sat_qps = len(sat_q) / sat["wall_s"]
        rows = []
        queries = synth.serving_queries(args.serve_queries, sizes, seed=7)
        for frac in args.serve_loads:
            rate = frac * sat_qps
            with ClockSampler(local) as clk:
                r = serve_phase(ctx, gids, alphas, queries, rate)
            rows.append({"load": frac, "offered_qps": rate, "achieved_qps": len(queries) / r["wall_s"],
                         "units_per_s": r["units"] / r["wall_s"], "p50_ms": percentile(r["latency_ms"], 50),
                         "p99_ms": percentile(r["latency_ms"], 99), "mean_ms": float(np.mean(r["latency_ms"])),
                         "queue_p50_ms": percentile(r["queue_ms"], 50), "queue_p99_ms": percentile(r["queue_ms"], 99),
                         "queries": len(queries), "clocks": clk.summary()})
        st = ctx.serve_stats()
        launches = L.mscd_launch_count() - l0
    finally:
        ctx.serve_stop()
    mid = rows[len(rows) // 2] if rows else None
    line = {"metric": "served local-community queries: p50/p99 latency and throughput",
            "value": mid["p99_ms"] if mid else None, "unit": "ms (p99 at %g of saturation)" % (mid["load"] if mid else 0),
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "dtype": "int64+f64",
            "config": {"workload": "serving: %d resident LFR-style graphs of %d nodes (mean degree 25, max 250, three "
                                   "levels, mixing 0.3/0.2/0.1, unweighted); Poisson queries, each on a uniform "
                                   "graph with 1-4096 uniform seeds at one of 16 log-spaced scales in [0.5,1]"
                                   % (len(graphs), sizes[0]),
                       "nnz": [g.nnz for g in graphs], "workers": args.serve_workers,
                       "max_batch_units": args.serve_batch_units},
            "saturation": {"queries": len(sat_q), "qps": sat_qps, "units_per_s": sat["units"] / sat["wall_s"],
                           "p50_ms": percentile(sat["latency_ms"], 50), "p99_ms": percentile(sat["latency_ms"], 99)},
            "loads": rows, "server_stats": st, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    ctx.close()


def read_results(ctx, n_scales, n_parts):
    """Device->host read of every scale's communities and every part's
    stability; returns the bytes read."""
    nb = 0
    for s in range(n_scales):
        ptr, nodes, f, s2c = ctx.communities(s)
        nb += ptr.nbytes + nodes.nbytes + f.nbytes + s2c.nbytes
    for p in range(n_parts):
        nmi, w3, w5 = ctx.stability(part=p)
        nb += nmi.nbytes + w3.nbytes + w5.nbytes
    return nb


class ServeSample:
    """Reference arm of the serving workload: the oracle answers queries of the
    same stream one after another (growth from every seed of the query)."""

    name = "serve"

    def __init__(self, args):
        import multiprocessing as mp

        from paper_1301_0955_gb300 import synth

        specs = synth.serving_specs(scale_nodes=args.serve_node_scale)
        with mp.get_context("spawn").Pool(len(specs)) as pool:
            self.graphs = pool.map(synth.graph_from_spec, specs, chunksize=1)
        import oracle

        rc, self.alphas = oracle.scales_logspaced(0.5, 1.0, 16)
        self.queries = synth.serving_queries(args.serve_queries, [g.n for g in self.graphs], seed=7)

    def config(self):
        return {"workload": "serving: %d resident LFR-style graphs of %d nodes, Poisson queries with 1-4096 seeds "
                            "at one of 16 scales (the oracle answers a prefix of the stream in turn)"
                            % (len(self.graphs), self.graphs[0].n)}

    def cpu_baseline(self, seconds, threads):
        import oracle

        Gs = [oracle.Graph(g.n, g.row_ptr, g.col) for g in self.graphs]
        units = 0
        dt = 0.0
        k = 0
        lat = []
        for g, s, seeds in self.queries:
            t0 = time.perf_counter()
            oracle.run(Gs[g], np.array([self.alphas[s]]), seeds, threads=threads)
            t = time.perf_counter() - t0
            lat.append(t * 1e3)
            dt += t
            units += len(seeds)
            k += 1
            if dt >= seconds:
                break
        return {"value": units / dt, "unit": "units/s", "cores": threads, "kind": "oracle",
                "sample": "the first %d queries of the stream (%d seeds), answered one after another by the "
                          "oracle on %d host threads, %.1f s; median query %.0f ms" % (k, units, threads, dt,
                                                                                     float(np.median(lat)))}


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    import oracle

    if args.workload not in WORKLOADS and args.workload != "serve":
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm covers the lfr-100k, "
                          "uneven-batch and serve workloads (the oracle on a bounded sample)"}), flush=True)
        return
    # the oracle's own scale list: this arm never loads the CUDA library
    def scales(vmin, a, x):
        rc, out = oracle.scales_logspaced(vmin, a, x)
        if rc != 0:
            raise RuntimeError("orc_scales_logspaced returned %d" % rc)
        return out

    wl = ServeSample(args) if args.workload == "serve" else WORKLOADS[args.workload](args, scales)
    threads = os.cpu_count() or 1
    per_step = max(1.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        wl.cpu_baseline(per_step / 4, threads)
    vals = [wl.cpu_baseline(per_step, threads) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    cfg = wl.config()
    cfg["sample"] = vals[-1]["sample"]
    line = {"impl": "reference", "metric": "seed expansions/s", "value": v, "unit": "units/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64+f128", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "units/s", "cores": threads, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "units/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "full":
        run_full(args)
        return
    if args.workload == "accuracy":
        run_accuracy(args)
        return
    world, rank, local = dist_env()
    from paper_1301_0955_gb300 import build, mscd

    build.build()  # nvcc only, no GPU call
    L = mscd.load()
    wl = WORKLOADS[args.workload](args, mscd.scales_logspaced)  # host-side generation before the first GPU call
    import torch

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = mscd.Context(local)
    stream = torch.cuda.current_stream(dev)
    wl.to_device(torch, dev)
    flush = torch.empty(max(1, args.flush_mib) * 256 * 1024, dtype=torch.int32, device=dev)  # > L2 (129 MB)
    units = wl.units

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def timed(step, k, c):
        times = []
        stats = []
        launches = 0
        out = None
        for _ in range(k):
            flush.zero_()
            barrier()
            l0 = L.mscd_launch_count()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = step(c)
            e1.record(stream)
            barrier()
            launches += L.mscd_launch_count() - l0
            times.append(e0.elapsed_time(e1))
            stats.append(c.run_stats())
        return times, stats, launches, out

    resident = lambda c: wl.step_resident(c, stream)  # noqa: E731
    for _ in range(args.warmup):
        resident(ctx)
    barrier()
    with ClockSampler(local) as clk:
        times, stats, launches, _ = timed(resident, args.steps, ctx)
    total_ms = reduce_max(sum(times), world)
    value = whole_job_rate(units, args.steps, world, total_ms)
    st = stats[-1]
    grow_ms = statistics.mean(s["ms_grow"] for s in stats)
    # algorithmic bytes: every scanned CSR entry (column, plus the exact weight
    # on a weighted graph) and the two row offsets of every row visited
    alg_bytes = (float(wl.bytes_per_entry) * st["edges_scanned"]
                 + 16.0 * (st["units"] + st["adds"] + st["removes"]))
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (grow_ms / 1e3) / 1e9
    traffic = None
    try:
        # only a capture of this kernel source on this exact unit set
        prof = json.load(open(PROFILE_FILES[wl.name]))
        if (prof.get("source_hash") == source_hash() and prof.get("workload") == wl.name
                and prof.get("units") == units):
            traffic = prof.get("dram_bytes_per_step")
    except Exception:
        pass
    # the plain GPU form: the same kernel, one launch per scale and slot
    # class, one statically mapped unit per warp (no persistence, no stealing)
    plain = None
    if args.plain_steps > 0:
        ctx_p = mscd.Context(local, schedule=mscd.SCHED_PER_SCALE)
        plain_step = lambda c: wl.step_plain(c, stream)  # noqa: E731
        plain_step(ctx_p)
        pt, pst, _, _ = timed(plain_step, args.plain_steps, ctx_p)
        p_ms = reduce_max(sum(pt), world) / args.plain_steps
        plain = {"schedule": "one launch per scale and slot class, one unit per warp"
                             + (", graph after graph" if wl.name == "uneven-batch" else ""),
                 "ms_per_step": p_ms, "value": whole_job_rate(units, 1, world, p_ms),
                 "steps": args.plain_steps, "speedup_step": p_ms / (total_ms / args.steps)}
        if wl.name != "uneven-batch":
            p_grow = statistics.mean(x["ms_grow"] for x in pst)
            plain.update({"ms_grow": p_grow, "grow_launches": pst[-1]["grow_launches"],
                          "speedup_grow": p_grow / grow_ms})
        ctx_p.close()
    e2e = None
    if not args.no_e2e:
        # the resident warm-up steps already ran every kernel and allocation;
        # a short workload also warms the host path once
        step_s = total_ms / args.steps / world / 1e3
        if step_s < 10.0:
            wl.step_e2e(ctx)
        et, _, _, d2h = timed(lambda c: wl.step_e2e(c), 1 if step_s >= 10.0 else max(1, min(args.steps, 2)), ctx)
        e2e = {"value": units / (statistics.mean(et) / 1e3), "unit": "units/s",
               "h2d_bytes_per_step": wl.h2d_bytes, "d2h_bytes_per_step": int(d2h),
               "ms_per_step": statistics.mean(et)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and getattr(wl, "full", True):
        cpu = wl.cpu_baseline(args.cpu_seconds, os.cpu_count() or 1)
        if isinstance(wl, SingleGraph):
            # the same oracle on one host thread, on a smaller adaptive sample
            one = wl.cpu_baseline(max(2.0, args.cpu_seconds / 3), 1)
            cpu["single_thread"] = {"value": one["value"], "unit": one["unit"], "sample": one["sample"]}
    if rank == 0:
        cfg = wl.config()
        cfg.update({"units_per_step_per_gpu": units, "l2": "flushed between steps (%d MiB write)" % args.flush_mib,
                    "parallelism": "replicas" if world > 1 else "single"})
        line = {
            "metric": "seed expansions/s", "value": value, "unit": "units/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
            "config": cfg,
            "edges_scanned_per_s": world * st["edges_scanned"] * args.steps / (total_ms / 1e3),
            "stage_ms": {k: st[k] for k in ("ms_grow", "ms_dedup", "ms_stability", "ms_total")},
            "run_stats": {k: st[k] for k in ("units", "edges_scanned", "adds", "removes", "slow_decisions",
                                             "undecided", "overflow_units", "grow_launches", "member_entries")},
            "roofline": {"bound": "hbm", "kernel": "grow_kernel", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_step": alg_bytes, "kernel_ms_per_step": grow_ms},
            "cpu_baseline": cpu,
            "plain_per_scale": plain,
            "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
