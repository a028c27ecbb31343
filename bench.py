#!/usr/bin/env python3
"""Benchmark of exact betweenness centrality (Brandes) on one GB300.

Metric: BC GTEPS = (sources x canonical edges) / seconds.  One step is one
complete BC job over the workload's source list (forward BFS with path
counts, backward dependency sweep, BC accumulation, output scaling) through
the library's C ABI with inputs resident in HBM; the `e2e` figure repeats the
step through the same C ABI starting from host buffers (graph upload, compute,
result download).  `precision` states the run's error against the FP64 CPU
oracle: the sources the CPU baseline timed are run again in the timed batch
width with FP32 and FP64 dependencies and compared element by element.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl ours|reference]

Under torchrun (N > 1) the workload's sources are split into N contiguous
shards, each rank computes its shard's partial BC and the partial vectors are
summed onto rank 0 (the one exchange step of the method).  `--impl reference`
times the CPU oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bcgen  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20

WORKLOADS = {
    # R-MAT scale 16, edge factor 16, all 65,536 sources (the library picks the batch width)
    "rmat16-exact": dict(kind="rmat", scale=16, ef=16, seed=1, sources="all", batch_k=0,
                         schedule="batch"),
    # R-MAT scale 20, edge factor 16, 4096 / 1024 seeded uniform sources
    "rmat20-sampled4096": dict(kind="rmat", scale=20, ef=16, seed=1, sources=4096,
                               src_seed=1, batch_k=0, schedule="batch"),
    "rmat20-sampled1024": dict(kind="rmat", scale=20, ef=16, seed=1, sources=1024,
                               src_seed=1, batch_k=0, schedule="batch"),
    # a smaller R-MAT case of the same recipe for detailed profiles (scale 18,
    # 1024 sources, four batches of 256; about 1.5 GB on the device)
    "rmat18-sampled1024": dict(kind="rmat", scale=18, ef=16, seed=1, sources=1024,
                               src_seed=1, batch_k=0, schedule="batch"),
    # directed preferential attachment n = 2^20, 8 out-edges, 4096 sources
    "ba20-sampled4096": dict(kind="ba", n=1 << 20, out=8, seed=1, sources=4096, src_seed=1,
                             batch_k=0, schedule="batch"),
    # the paper's largest input: undirected preferential attachment, n = 30,000,
    # 30 edges per arrival stored both ways (edge density m/n = 60), all sources
    "ba30k-d60-exact": dict(kind="ba_undirected", n=30000, beta=30, seed=1, sources="all",
                            batch_k=0, schedule="batch"),
    # R-MAT scale 10, edge factor 8, all 1024 sources, one source per launch
    "rmat10-exact-plain": dict(kind="rmat", scale=10, ef=8, seed=1, sources="all", batch_k=1,
                               schedule="plain", fp64=True),
}


def make_graph(w):
    if w["kind"] == "rmat":
        return bcgen.rmat(w["scale"], w["ef"], seed=w["seed"])
    if w["kind"] == "ba_undirected":
        return bcgen.ba_undirected(w["n"], w["beta"], seed=w["seed"])
    return bcgen.ba_directed(w["n"], w["out"], 9, seed=w["seed"])


def source_list(w, n):
    if w["sources"] == "all":
        return np.arange(n, dtype=np.int32)
    return bcgen.sample_sources(n, w["sources"], seed=w["src_seed"])


def describe(name, w, g, nsrc):
    d = {"workload": name, "graph": g.name, "n": g.n, "m": g.m, "sources": nsrc,
         "batch_k": w["batch_k"], "schedule": w["schedule"]}
    return d


# ---- bytes model --------------------------------------------------------------

def bytes_model(stats, delta_bytes):
    """Design bytes model: algorithmic bytes of the BC kernels as this design
    lays out its data, for the counters of one job (element granularity, each
    element the design must touch counted once; b = bytes of one dependency
    value, W = 64-bit words per source mask).

    queue batch kernel (kernel_kind 2): 124 B per frontier entry (queue
           id/mask, CSR offsets, dense mask read/write/clear, visited, BC),
           4 + 8W B per scanned edge (the neighbour id and its W-word mask),
           (8 + b) B per (source, DAG edge) (predecessor path count,
           successor coefficient), (16 + b) B per (source, reached vertex)
           (path count write and read, coefficient write; the reset of each
           count after its backward step is not counted).
    plain kernel (1): (84 + b) B per entry, 8 B per scanned edge (column +
           int32 depth), (8 + b) B per DAG edge.
    """
    E = stats["frontier_entries"]
    I, O = stats["scanned_in_edges"], stats["scanned_out_edges"]
    D, R = stats["dag_pairs"], stats["reached_pairs"]
    b = delta_bytes
    if stats.get("kernel_kind", 2) == 2:
        W = max(int(stats.get("mask_words") or 1), 1)
        return 124 * E + (4 + 8 * W) * (I + O) + (8 + b) * D + (16 + b) * R
    return (84 + b) * E + 8 * (I + O) + (8 + b) * D


def method_bytes_model(stats, delta_bytes):
    """The method's bytes model, independent of this design's layout, per
    job: every element the batched sweeps must touch, at the width the method
    states it.  Batched, k sources per batch: the CSR once per batch and level (8 B of
    offsets per frontier entry, 4 B per scanned edge), k/8 B of source
    bitset per scanned edge endpoint, per (source, DAG edge) a 16-byte path
    count read-modify-write and a b-byte coefficient read, per (source,
    reached vertex) 16 + b bytes of count, dependency and BC terms:
        8 E + 4 (I + O) + (k/8)(I + O) + (16 + b) D + (16 + b) R.
    One source per launch (plain): 8 B per scanned edge (column + depth
    test), (24 + b) B per DAG edge, (72 + 2b) B per reached vertex:
        8 (I + O) + (24 + b) D + (72 + 2b) E."""
    E = stats["frontier_entries"]
    I, O = stats["scanned_in_edges"], stats["scanned_out_edges"]
    D, R = stats["dag_pairs"], stats["reached_pairs"]
    b = delta_bytes
    if stats.get("kernel_kind", 2) == 2:
        k = 64 * max(int(stats.get("mask_words") or 1), 1)
        return 8 * E + 4 * (I + O) + (k // 8) * (I + O) + (16 + b) * D + (16 + b) * R
    return 8 * (I + O) + (24 + b) * D + (72 + 2 * b) * E


KERNEL_NAMES = {1: "plain_kernel", 2: "batch_kernel"}
METHOD_MODEL_TEXT = {2: "8E + 4(I+O) + (k/8)(I+O) + (16+b)D + (16+b)R, k = 64 x mask_words",
                     1: "8(I+O) + (24+b)D + (72+2b)E"}
DESIGN_MODEL_TEXT = {2: "124E + (4+8W)(I+O) + (8+b)D + (16+b)R, W = mask_words",
                     1: "(84+b)E + 8(I+O) + (8+b)D"}


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ["bc_kernels.cu", "bc_narrow.cu", "bc_batch.cuh", "bc_device.cuh", "bc_internal.cuh"]:
        with open(os.path.join(ROOT, "paper_1409_7764_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per launch of the batch kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    entry = rec.get(workload)
    if not entry or entry.get("kernel_sha") != kernel_source_sha():
        return None
    return entry.get("dram_bytes_per_launch")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback"


# ---- clocks -------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        # raw samples: kept in BENCH_CLOCKS_DIR if set, else a temporary file
        self.keep = bool(os.environ.get("BENCH_CLOCKS_DIR"))
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"bench_clocks_dev{device}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        if not self.keep:
            try:
                os.remove(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- CPU oracle baseline ----------------------------------------------------------

def _oracle_chunk(args):
    n, rp, ci, srcs = args[:4]
    keep = len(args) > 4 and args[4]
    import oracle
    bc, _ = oracle.bc(n, rp, ci, srcs)
    return (len(srcs), bc) if keep else len(srcs)


def cpu_oracle_run(pool, cores, g, srcs, target_s, keep_bc=False):
    """Times the oracle (as it stands) on a bounded sample of the workload's
    sources, split over `cores` spawned worker processes.  With keep_bc the
    oracle's BC over the sample is returned too (key "bc", "sample_sources")."""
    import oracle
    t0 = time.perf_counter()
    oracle.bc(g.n, g.row_ptr, g.col_idx, srcs[:1])
    t1 = max(time.perf_counter() - t0, 1e-4)
    count = int(max(cores, min(len(srcs), target_s * cores / t1)))
    sample = srcs[:count]
    parts = [(g.n, g.row_ptr, g.col_idx, s, keep_bc) for s in np.array_split(sample, cores)
             if len(s)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_chunk, parts)
    wall = time.perf_counter() - t0
    done = sum(r[0] for r in res) if keep_bc else sum(res)
    out = {"value": done * g.m / wall / 1e9, "unit": "GTEPS", "cores": len(parts),
           "kind": "oracle",
           "sample": f"first {done} of the workload's {len(srcs)} sources "
                     f"(sequential Brandes in C, one process per core)",
           "seconds": wall}
    if keep_bc:
        bc = np.zeros(g.n)
        for r in res:  # fixed order: the partial sums of consecutive source ranges
            bc += r[1]
        out["bc"] = bc
        out["sample_sources"] = sample
    return out


def rel_errors(got, ref):
    """Max and 99th-percentile relative error where the reference is not 0,
    and whether the reference's exact zeros are exact zeros."""
    got, ref = np.asarray(got), np.asarray(ref)
    zero = ref == 0
    nz = ~zero
    rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz]) if nz.any() else np.zeros(1)
    return {"max_rel": float(rel.max()), "p99_rel": float(np.percentile(rel, 99)),
            "zeros_exact": bool(np.array_equal(got[zero], ref[zero]))}


# ---- reference arm ------------------------------------------------------------------

def run_reference(args, w, name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g = make_graph(w)
    srcs = source_list(w, g.n)
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk, [(g.n, g.row_ptr, g.col_idx, srcs[:1])] * cores)
        per_step_target = 6.0
        res = []
        for i in range(args.warmup + args.steps):
            r = cpu_oracle_run(pool, cores, g, srcs, per_step_target)
            if i >= args.warmup:
                res.append(r)
    vals = [r["value"] for r in res]
    value = statistics.mean(vals)
    secs = [r["seconds"] for r in res]
    line = {
        "impl": "reference", "metric": "BC GTEPS (sources*m/s)", "value": value,
        "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(secs), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
        "config": describe(name, w, g, len(srcs)),
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": res[0]["cores"],
                         "kind": "oracle", "sample": res[0]["sample"]},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- our arm ----------------------------------------------------------------------

def run_ours(args, w, name):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    g = make_graph(w)
    srcs = source_list(w, g.n)
    if args.max_sources:
        srcs = srcs[:args.max_sources]
    from paper_1409_7764_gb300.sharding import reduce_partial_bc, shard_sources
    mine = shard_sources(srcs, world, rank)

    pool = None
    cores = os.cpu_count() or 1
    if rank == 0 and not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(cores)  # before any GPU call
        pool.map(_oracle_chunk, [(g.n, g.row_ptr, g.col_idx, srcs[:1])] * cores)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_1409_7764_gb300 as bc
    stream = torch.cuda.current_stream()
    ctx = bc.Context(local, stream=stream)
    fp64 = bool(w.get("fp64", False)) or args.fp64
    opts = dict(schedule=args.schedule or w["schedule"], batch_k=w["batch_k"],
                delta_fp64=fp64, keep_source_order=args.keep_source_order,
                count_bits=args.count_bits, direction=args.direction)
    G = ctx.create_graph(g.row_ptr, g.col_idx)
    out = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step():
        ctx.sources(G, mine, out=out, **opts)
        if dist is not None:
            reduce_partial_bc(out, dist, dst=0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = []
    stats = []
    for _ in range(args.steps):
        flush.fill_(1)  # L2 flush between timed steps (outside the events)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        step()
        e.record(stream)
        evs.append((s, e))
        stats.append(ctx.last_stats())
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in evs]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = len(srcs) * g.m / (ms_per_step / 1e3) / 1e9

    # kernel-level roofline of the batch (or plain) kernel on this rank
    st = stats[-1]
    delta_bytes = 8 if fp64 else 4
    algo_bytes = method_bytes_model(st, delta_bytes)
    design_bytes = bytes_model(st, delta_bytes)
    launches = max(st["batches"], 1)
    my_ms = sum(step_ms) / args.steps
    achieved = algo_bytes / (my_ms / 1e3) / 1e9
    design_achieved = design_bytes / (my_ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    traffic = ncu_traffic(name)

    # end-to-end: host CSR in (pinned host memory), host BC out (pinned), through
    # the C ABI: graph creation (validation, upload, device-side preparation),
    # the job, the result copy and the graph's release, every step
    e2e_ms = []
    e2e_steps = 0 if args.skip_e2e else args.steps + 1
    pin_rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int32)).pin_memory()
    pin_ci = torch.from_numpy(np.ascontiguousarray(g.col_idx, dtype=np.int32)).pin_memory()
    pin_out = torch.empty(g.n, dtype=torch.float64).pin_memory()
    rp_h, ci_h, host_out = pin_rp.numpy(), pin_ci.numpy(), pin_out.numpy()
    for i in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = ctx.create_graph(rp_h, ci_h)
        ctx.sources(G2, mine, out=host_out, **opts)
        ctx.destroy_graph(G2)
        t1 = time.perf_counter()
        if i > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_step = statistics.mean(e2e_ms) if e2e_ms else float("nan")
    if dist is not None:
        t = torch.tensor([e2e_step], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step = float(t.item())
    e2e_value = len(srcs) * g.m / (e2e_step / 1e3) / 1e9 if e2e_ms else None
    h2d = 4 * (g.n + 1) + 4 * g.m + (0 if w["sources"] == "all" else 4 * len(mine))
    d2h = 8 * g.n

    extra = {}
    if rank == 0 and not args.quick:
        # the plain one-source-per-launch path on a sample of the same sources
        if opts["schedule"] != "plain":
            sample = mine[:min(len(mine), args.plain_sample)]
            ctx.sources(G, sample[:4], out=out, schedule="plain", delta_fp64=fp64)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            ctx.sources(G, sample, out=out, schedule="plain", delta_fp64=fp64)
            e.record(stream)
            torch.cuda.synchronize()
            pms = s.elapsed_time(e)
            extra["plain"] = {"value": len(sample) * g.m / (pms / 1e3) / 1e9, "unit": "GTEPS",
                              "sources": int(len(sample)),
                              "note": "one source per launch, same graph and sources"}
            # the other dependency precision on the same job
            s.record(stream)
            ctx.sources(G, mine, out=out, **dict(opts, delta_fp64=not fp64))
            e.record(stream)
            torch.cuda.synchronize()
            oms = s.elapsed_time(e)
            extra["fp64_delta" if not fp64 else "fp32_delta"] = {
                "value": len(srcs) * g.m / (oms / 1e3) / 1e9, "unit": "GTEPS"}

    cpu = None
    precision = None
    if pool is not None:
        cpu = cpu_oracle_run(pool, cores, g, srcs, args.cpu_seconds, keep_bc=True)
        pool.close()
        cpu.pop("seconds", None)
        # the run's error against the FP64 oracle: the same sampled sources in
        # the timed run's batch width, with FP32 and FP64 dependencies
        ref_bc, sample = cpu.pop("bc"), cpu.pop("sample_sources")
        kb = int(st.get("batch_sources") or 0)
        precision = {"sources": int(len(sample)), "reference": "CPU oracle (FP64 dependencies)"}
        for name_, f64 in (("fp32_delta", False), ("fp64_delta", True)):
            ctx.sources(G, sample, out=out, **dict(opts, delta_fp64=f64, batch_k=kb))
            precision[name_] = rel_errors(out.cpu().numpy(), ref_bc)

    if rank == 0 and not args.quick and args.line_serve_requests > 0:
        # the serving loop at stated load, compactly: 2 seeds per scale in the
        # graph pool, line_serve_requests requests per offered load
        extra["serving"] = serving_experiment(ctx, args.line_serve_requests, [1, 2],
                                              args.serve_seed)

    if rank == 0:
        line = {
            "metric": "BC GTEPS (sources*m/s)", "value": value, "unit": "GTEPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None,
            "dtype": ("u64" if (args.count_bits == 64 or opts["schedule"] == "plain") else "u32")
                     + ("+f64" if fp64 else "+f32"),
            "data": "synthetic",
            "config": dict(describe(name, w, g, len(srcs)),
                           batch_k=int(st.get("batch_sources") or w["batch_k"]),
                           l2="flushed between timed steps (512 MiB write)",
                           parallelism=f"source shards x{world}",
                           source_order="given" if args.keep_source_order
                           else "grouped (library batch composition)"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "kernel": KERNEL_NAMES.get(st.get("kernel_kind"), "?"),
                         "model": METHOD_MODEL_TEXT.get(st.get("kernel_kind"), "?"),
                         "algo_bytes_per_launch": algo_bytes / launches,
                         "launch_ms": my_ms / launches,
                         "design_model": {
                             "formula": DESIGN_MODEL_TEXT.get(st.get("kernel_kind"), "?"),
                             "bytes_per_launch": design_bytes / launches,
                             "achieved": design_achieved, "frac": design_achieved / peak}},
            "cpu_baseline": cpu,
            "precision": precision,
            "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(st["kernel_launches"]) * args.steps,
            "clocks": clk,
            "counters": {k: st[k] for k in ("frontier_entries", "scanned_in_edges",
                                            "scanned_out_edges", "dag_pairs", "reached_pairs",
                                            "heavy_chunks", "max_levels", "levels_sum",
                                            "batches", "kernel_kind", "chunk_edges", "grab",
                                            "batch_sources", "mask_words", "push_levels",
                                            "batch_groups")},
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# ---- many small graphs in one launch ----------------------------------------------

def many_graphs(count, seed=1):
    """`count` R-MAT graphs, scale uniform in [6, 12], edge factor uniform in
    [4, 16], graph i seeded by splitmix64(seed ^ i)."""
    return [bcgen.rmat(s, ef, sd) for s, ef, sd in bcgen.small_rmat_specs(count, master_seed=seed)]


def _oracle_graphs(args):
    import oracle
    done = 0
    for n, rp, ci in args:
        oracle.bc(n, rp, ci)
        done += 1
    return done


def run_many(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    graphs = many_graphs(args.many_count)
    work = sum(g.n * g.m for g in graphs)
    cores = os.cpu_count() or 1
    pool = None
    if not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(cores)
        pool.map(_oracle_chunk, [(graphs[0].n, graphs[0].row_ptr, graphs[0].col_idx,
                                  np.arange(1, dtype=np.int32))] * cores)
    import torch
    import paper_1409_7764_gb300 as bc
    stream = torch.cuda.current_stream()
    ctx = bc.Context(0, stream=stream)
    fp64 = args.fp64
    hs = [ctx.create_graph(g.row_ptr, g.col_idx) for g in graphs]
    # the device-timed steps write BC to HBM (one vector); e2e below returns it to the host
    dev_out = torch.zeros(sum(g.n for g in graphs), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        ctx.exact_many(hs, out=dev_out, delta_fp64=fp64, keep_source_order=args.keep_source_order,
                       batch_k=max(args.batch_k, 0), count_bits=args.count_bits)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ms, stats = [], None
    for _ in range(args.steps):
        flush.fill_(1)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        ctx.exact_many(hs, out=dev_out, delta_fp64=fp64, keep_source_order=args.keep_source_order,
                       batch_k=max(args.batch_k, 0), count_bits=args.count_bits)
        e.record(stream)
        torch.cuda.synchronize()
        ms.append(s.elapsed_time(e))
        stats = ctx.last_stats()
    clk = clocks.stop()
    ms_step = statistics.mean(ms)
    value = work / (ms_step / 1e3) / 1e9
    algo = bytes_model(stats, 8 if fp64 else 4)
    peak, peak_kind = peaks()
    # end to end: host CSR in, host BC out, for all graphs
    e2e = []
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = ctx.create_graphs([(g.row_ptr, g.col_idx) for g in graphs])
        ctx.exact_many(h2, delta_fp64=fp64, batch_k=max(args.batch_k, 0),
                       count_bits=args.count_bits)
        for h in h2:
            ctx.destroy_graph(h)
        e2e.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e)
    cpu = None
    if pool is not None:
        # the oracle on the first graphs of the list, about cpu_seconds of work
        t0 = time.perf_counter()
        _oracle_graphs([(graphs[0].n, graphs[0].row_ptr, graphs[0].col_idx)])
        t1 = max(time.perf_counter() - t0, 1e-4)
        per = graphs[0].n * graphs[0].m
        budget = args.cpu_seconds * cores / t1 * per
        sample, acc = [], 0
        for g in graphs:
            if acc >= budget:
                break
            sample.append(g)
            acc += g.n * g.m
        parts = [[(g.n, g.row_ptr, g.col_idx) for g in sample[i::cores]] for i in range(cores)]
        t0 = time.perf_counter()
        pool.map(_oracle_graphs, [p for p in parts if p])
        wall = time.perf_counter() - t0
        pool.close()
        cpu = {"value": acc / wall / 1e9, "unit": "GTEPS", "cores": cores, "kind": "oracle",
               "sample": f"exact BC of the first {len(sample)} of the {len(graphs)} graphs, "
                         f"one process per core"}
    line = {
        "metric": "BC GTEPS (sources*m/s)", "value": value, "unit": "GTEPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": ("u64" if args.count_bits == 64 else "u32") + ("+f64" if fp64 else "+f32"),
        "data": "synthetic",
        "config": {"workload": "rmat-many10k", "graphs": len(graphs),
                   "scales": "6..12 uniform", "edge_factors": "4..16 uniform",
                   "sum_n": int(sum(g.n for g in graphs)), "sum_m": int(sum(g.m for g in graphs)),
                   "l2": "flushed between timed steps (512 MiB write)",
                   "schedule": "one persistent launch, one block per graph, "
                               + (f"{args.batch_k} sources per batch" if args.batch_k > 0
                                  else "64, 128 or 256 sources per batch by graph size")},
        "roofline": {"bound": "hbm", "achieved": algo / (ms_step / 1e3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": algo / (ms_step / 1e3) / 1e9 / peak,
                     "traffic": None, "peak_kind": peak_kind, "kernel": "many_kernel"},
        "cpu_baseline": cpu,
        "e2e": {"value": work / e2e_s / 1e9, "unit": "GTEPS",
                "h2d_bytes_per_step": int(sum(4 * (g.n + 1) + 4 * g.m for g in graphs)),
                "d2h_bytes_per_step": int(sum(8 * g.n for g in graphs))},
        "gpu_launches": int(stats["kernel_launches"]) * args.steps,
        "clocks": clk,
        "counters": {k: stats[k] for k in ("frontier_entries", "scanned_in_edges",
                                           "scanned_out_edges", "dag_pairs", "reached_pairs",
                                           "heavy_chunks", "max_levels", "batches")},
    }
    print(json.dumps(line), flush=True)
    ctx.close()


# ---- serving ----------------------------------------------------------------------

def serving_experiment(ctx, n_requests, seeds, serve_seed):
    """Open-loop serving of BC requests on a pool of device-resident R-MAT
    graphs (scales 8..20, edge factor 16, one per seed and scale): exact BC
    up to scale 14, 1024 seeded sampled sources above.  Capacity comes from
    solo service times; at offered loads rho = 0.5 and 0.8 of it, the same
    Poisson request stream runs with FP32 and then FP64 dependencies, so the
    FP32 results can be compared with the FP64 ones request by request."""
    from paper_1409_7764_gb300.serving import (Request, poisson_arrivals, run_open_loop,
                                                solo_service_times, summarize)
    scales = list(range(8, 21))
    pool = {}
    for sc in scales:
        for sd in seeds:
            g = bcgen.rmat(sc, 16, seed=sd)
            pool[(sc, sd)] = ctx.create_graph(g.row_ptr, g.col_idx)
    rs = np.random.default_rng(serve_seed)

    def make_requests(count):
        reqs = []
        for i in range(count):
            sc = int(rs.integers(8, 21))
            G = pool[(sc, seeds[int(rs.integers(0, len(seeds)))])]
            srcs = None if sc <= 14 else bcgen.sample_sources(G.n, 1024, seed=1000 + i)
            reqs.append(Request(G, srcs, {}))
        return reqs

    def with_opts(reqs, fp64):
        return [Request(r.graph, r.sources, dict(delta_fp64=fp64)) for r in reqs]

    out = {"fp32": {}, "fp64": {}, "fp32_vs_fp64": {}}
    taus = {}
    for fp64 in (False, True):
        probe = [Request(pool[(sc, seeds[0])],
                         None if sc <= 14 else bcgen.sample_sources(pool[(sc, seeds[0])].n, 1024,
                                                                    seed=7),
                         dict(delta_fp64=fp64)) for sc in scales]
        solo_service_times(ctx, probe[:3])  # warm-up
        tau = float(np.mean(solo_service_times(ctx, probe)))
        taus[fp64] = tau
        key = "fp64" if fp64 else "fp32"
        out[key]["mean_solo_ms"] = tau * 1e3
        out[key]["capacity_rps"] = 1.0 / tau
    for rho in (0.5, 0.8):
        reqs = make_requests(n_requests)
        got = {}
        for fp64 in (False, True):
            arr = poisson_arrivals(len(reqs), rho / taus[fp64], seed=serve_seed + int(rho * 10))
            results = {}
            recs = run_open_loop(ctx, with_opts(reqs, fp64), arr, results=results)
            out["fp64" if fp64 else "fp32"][f"rho{rho}"] = summarize(recs)
            got[fp64] = results
        # each request's FP32 result against its FP64 result
        worst = []
        for i, r64 in got[True].items():
            r32 = got[False].get(i)
            if r32 is None or r64 is None:
                continue
            nz = r64 != 0
            worst.append(float(np.max(np.abs(r32[nz] - r64[nz]) / np.abs(r64[nz])))
                         if nz.any() else 0.0)
        out["fp32_vs_fp64"][f"rho{rho}"] = {
            "requests": len(worst), "max_rel": max(worst) if worst else None,
            "p99_rel": float(np.percentile(worst, 99)) if worst else None}
    for G in pool.values():
        ctx.destroy_graph(G)
    out["pool"] = f"R-MAT scales 8..20 x {len(seeds)} seeds, edge factor 16"
    out["request_mix"] = "scale uniform 8..20; exact for scale <= 14, 1024 seeded sources above"
    out["arrivals"] = "Poisson at rho x capacity (capacity from solo service times)"
    return out


def run_serving(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import paper_1409_7764_gb300 as bc
    ctx = bc.Context(0)
    out = serving_experiment(ctx, args.serve_requests, [1, 2, 3, 4], args.serve_seed)
    main = out["fp32"]["rho0.8"]
    line = {
        "metric": "BC GTEPS (sources*m/s)", "value": main["gteps"], "unit": "GTEPS", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u64+f32", "data": "synthetic",
        "config": {"workload": "serving", "requests": args.serve_requests,
                   "pool": out["pool"], "request_mix": out["request_mix"],
                   "arrivals": out["arrivals"]},
        "serving": out,
        "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat20-sampled4096",
                    choices=sorted(WORKLOADS) + ["rmat-many10k", "serving"])
    ap.add_argument("--fp64", action="store_true", help="FP64 dependencies")
    ap.add_argument("--plain-sample", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the plain / precision extras")
    ap.add_argument("--skip-e2e", action="store_true",
                    help="no end-to-end steps (profiling runs: the timed job's launches come last)")
    ap.add_argument("--schedule", default=None,
                    choices=["plain", "batch", "batch_queue"],
                    help="override the workload's schedule")
    ap.add_argument("--max-sources", type=int, default=0,
                    help="use only the first N sources of the workload (profiling runs)")
    ap.add_argument("--batch-k", type=int, default=-1,
                    help="sources per batch (0: the library picks; default: the workload's)")
    ap.add_argument("--keep-source-order", action="store_true",
                    help="batches take the sources in the given order instead of the library's grouping")
    ap.add_argument("--count-bits", type=int, default=0, choices=[0, 32, 64],
                    help="path-count storage (0: the library's default, 32 bits with promotion)")
    ap.add_argument("--direction", default="auto", choices=["auto", "pull", "push"],
                    help="path-count step direction of the batched forward levels")
    ap.add_argument("--many-count", type=int, default=10000)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--line-serve-requests", type=int, default=500,
                    help="requests per offered load of the serving record in the main line "
                         "(0: none)")
    ap.add_argument("--serve-seed", type=int, default=1)
    args = ap.parse_args()
    if args.workload == "rmat-many10k" and args.impl == "ours":
        return run_many(args)
    if args.workload == "serving" and args.impl == "ours":
        return run_serving(args)
    if args.workload in ("rmat-many10k", "serving"):
        print(json.dumps({"impl": "reference",
                          "unavailable": "the reference arm covers the single-graph workloads"}))
        return
    w = WORKLOADS[args.workload]
    if args.batch_k >= 0:
        w = dict(w, batch_k=args.batch_k)
    if args.impl == "reference":
        run_reference(args, w, args.workload)
    else:
        run_ours(args, w, args.workload)


if __name__ == "__main__":
    main()
