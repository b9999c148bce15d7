#!/usr/bin/env python
"""Benchmark of the multi-scale LFK community-growth hot path on one GB300.

Workload (one step): the 100,000-node LFR-style hierarchical graph (power-law
degrees tau = 2.5, mean 20, max 200; community sizes 20..1000, tau = 1.5; two
levels; mixing 0.3 / 0.1; unweighted), 20 log-spaced scales in [0.5, 1],
every node a seed: graph checks and exact weights, growth of all 2,000,000
(scale, seed) units, dedup per scale, NMI between successive scales.

  value      seed expansions (units) per second, graph already resident in HBM
  e2e        the same through the C ABI from pinned host buffers, with the
             host->device copy of the graph and the device->host read of every
             scale's communities and the stability inside the timed region
  roofline   growth kernel: algorithmic bytes (4 B per CSR entry scanned +
             16 B per row visited) / growth time, against the measured HBM copy
             bandwidth

--impl reference times the CPU oracle (the reference arm of this build) on a
bounded sample of the same workload.  Under torchrun every rank runs its own
replica of the workload (weak scaling, no collective on the data path).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SCALES = 20
WORKLOAD = ("lfr-100k: 100,000-node LFR-style hierarchical graph (degrees power-law 2.5, mean 20, max 200; "
            "community sizes 20-1000 power-law 1.5; 2 levels, mixing 0.3/0.1; unweighted, seed 1), "
            "20 log-spaced scales in [0.5,1], every node a seed")
GROW_SOURCES = ["paper_1301_0955_gb300/csrc/grow.cu", "paper_1301_0955_gb300/csrc/exact.cuh",
                "paper_1301_0955_gb300/csrc/grow.cuh"]
PROFILE_FILE = os.path.join(ROOT, "profiles", "grow_kernel_lfr100k_traffic.json")
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
    p.add_argument("--scales", type=int, default=N_SCALES, help="profiling: fewer scales")
    p.add_argument("--flush-mib", type=int, default=1024, help="L2 flush buffer written between steps")
    p.add_argument("--plain-steps", type=int, default=1,
                   help="steps of the plain one-launch-per-scale form timed for comparison (0: skip)")
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
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench.csv")

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


def oracle_sample(g, alphas, seconds, threads):
    """Time the oracle (growth + dedup per scale) on a seeded sample of seeds
    at every scale, sized to about `seconds` of CPU time."""
    import oracle

    G = oracle.Graph(g.n, g.row_ptr, g.col, g.w)
    rng = np.random.default_rng(12345)
    m = 8
    while True:
        seeds = np.sort(rng.choice(g.n, m, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        rc, ptr, nodes, f, st = oracle.run(G, alphas, seeds, threads=threads)
        for s in range(len(alphas)):
            lo, hi = s * m, (s + 1) * m
            oracle.dedup(ptr[lo:hi + 1] - ptr[lo], nodes[ptr[lo]:ptr[hi]])
        dt = time.perf_counter() - t0
        if dt >= seconds * 0.5 or m >= g.n:
            break
        m = int(min(g.n, max(2 * m, m * seconds / max(dt, 1e-3) * 0.9)))
    units = m * len(alphas)
    return {"value": units / dt, "unit": "units/s", "cores": threads, "kind": "oracle",
            "sample": "%d seeds (seeded) x %d scales = %d units of the same workload, oracle growth + dedup on "
                      "%d host threads, %.1f s" % (m, len(alphas), units, threads, dt),
            "edges_scanned_per_s": float(st[:, 0].sum()) / dt}


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1301_0955_gb300 import synth

    g = synth.config_graph(1)
    rc, alphas = oracle.scales_logspaced(0.5, 1.0, N_SCALES)
    threads = os.cpu_count() or 1
    per_step = max(1.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(g, alphas, per_step / 4, threads)
    vals = [oracle_sample(g, alphas, per_step, threads) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    line = {"impl": "reference", "metric": "seed expansions/s", "value": v, "unit": "units/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64+f128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": vals[-1]["sample"]},
            "cpu_baseline": {"value": v, "unit": "units/s", "cores": threads, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "units/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1301_0955_gb300 import build, mscd, synth

    build.build()
    L = mscd.load()
    g = synth.config_graph(1)
    n_scales = args.scales
    alphas = mscd.scales_logspaced(0.5, 1.0, n_scales)
    seeds_h = None
    if args.seeds:
        seeds_h = np.sort(np.random.default_rng(0).choice(g.n, args.seeds, replace=False)).astype(np.int32)
    ctx = mscd.Context(local)
    stream = torch.cuda.current_stream(dev)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    alphas_d = torch.from_numpy(alphas).to(dev)
    seeds_d = None if seeds_h is None else torch.from_numpy(seeds_h).to(dev)
    flush = torch.empty(max(1, args.flush_mib) * 256 * 1024, dtype=torch.int32, device=dev)  # > L2 (129 MB)
    units = n_scales * (g.n if seeds_h is None else len(seeds_h))

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def step_resident():
        gid = ctx.load_csr(g.n, rp_d, col_d)
        rc = ctx.run(gid, alphas_d, seeds_d, stream=stream)
        assert rc == mscd.OK, rc
        ctx.free_graph(gid)

    # pinned host copies for the end-to-end path
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    rp_hn, col_hn = rp_h.numpy(), col_h.numpy()
    d2h_bytes = [0]

    def step_e2e():
        gid = ctx.load_csr(g.n, rp_hn, col_hn)
        rc = ctx.run(gid, alphas, seeds_h)
        assert rc == mscd.OK, rc
        nb = 0
        for s in range(n_scales):
            ptr, nodes, f, s2c = ctx.communities(s)
            nb += ptr.nbytes + nodes.nbytes + f.nbytes + s2c.nbytes
        nmi, w3, w5 = ctx.stability()
        nb += nmi.nbytes + w3.nbytes + w5.nbytes
        d2h_bytes[0] = nb
        ctx.free_graph(gid)

    def timed(step, k, c=ctx):
        times = []
        stats = []
        launches = 0
        for _ in range(k):
            flush.zero_()
            barrier()
            l0 = L.mscd_launch_count()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            barrier()
            launches += L.mscd_launch_count() - l0
            times.append(e0.elapsed_time(e1))
            stats.append(c.run_stats())
        return times, stats, launches

    for _ in range(args.warmup):
        step_resident()
    barrier()
    with ClockSampler(local) as clk:
        times, stats, launches = timed(step_resident, args.steps)
    total_ms = reduce_max(sum(times), world)
    value = whole_job_rate(units, args.steps, world, total_ms)
    st = stats[-1]
    grow_ms = statistics.mean(s["ms_grow"] for s in stats)
    alg_bytes = 4.0 * st["edges_scanned"] + 16.0 * (st["units"] + st["adds"] + st["removes"])
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (grow_ms / 1e3) / 1e9
    traffic = None
    try:
        prof = json.load(open(PROFILE_FILE))
        if prof.get("source_hash") == source_hash():
            traffic = prof.get("dram_bytes_per_step")
    except Exception:
        pass
    # the plain GPU form: the same kernel, one launch per scale and slot
    # class, one statically mapped unit per warp (no persistence, no stealing)
    plain = None
    if args.plain_steps > 0:
        ctx_p = mscd.Context(local, schedule=mscd.SCHED_PER_SCALE)

        def step_plain():
            gid = ctx_p.load_csr(g.n, rp_d, col_d)
            rc = ctx_p.run(gid, alphas_d, seeds_d, stream=stream)
            assert rc == mscd.OK, rc
            ctx_p.free_graph(gid)

        step_plain()
        pt, pst, _ = timed(step_plain, args.plain_steps, ctx_p)
        p_ms = reduce_max(sum(pt), world) / args.plain_steps
        p_grow = statistics.mean(x["ms_grow"] for x in pst)
        plain = {"schedule": "one launch per scale and slot class, one unit per warp",
                 "ms_per_step": p_ms, "value": whole_job_rate(units, 1, world, p_ms), "ms_grow": p_grow,
                 "grow_launches": pst[-1]["grow_launches"], "steps": args.plain_steps,
                 "speedup_step": p_ms / (total_ms / args.steps), "speedup_grow": p_grow / grow_ms}
        ctx_p.close()
    e2e = None
    if not args.no_e2e:
        step_e2e()  # warm the host path once
        et, _, _ = timed(step_e2e, max(1, min(args.steps, 2)))
        e2e = {"value": units / (statistics.mean(et) / 1e3), "unit": "units/s",
               "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col.nbytes + alphas.nbytes),
               "d2h_bytes_per_step": int(d2h_bytes[0]), "ms_per_step": statistics.mean(et)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and seeds_h is None:
        cpu = oracle_sample(g, alphas, args.cpu_seconds, os.cpu_count() or 1)
    if rank == 0:
        line = {
            "metric": "seed expansions/s", "value": value, "unit": "units/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if seeds_h is None and n_scales == N_SCALES else
                       "profiling subset: %d seeds x %d scales of the lfr-100k workload" % (units // n_scales, n_scales),
                       "n_nodes": g.n, "nnz": g.nnz, "scales": n_scales, "seeds": units // n_scales,
                       "units_per_step_per_gpu": units, "l2": "flushed between steps (%d MiB write)" % args.flush_mib,
                       "parallelism": "replicas" if world > 1 else "single"},
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
