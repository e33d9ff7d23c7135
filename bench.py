"""Benchmark: Monte Carlo edge-weighted PPR on one GB300 (or N independent replicas).

One step = one pass of the whole hot path over the workload: build the walk
layout from the device-resident CSR (node records, weight prefixes), run R
walks from every source with the persistent walker, and aggregate the
endpoints into sparse count rows and top-k.  The metric is walk steps per
second (draws consumed); walks per second and the roofline of the walker
kernel are reported beside it.

Default workload: R-MAT scale 24 (16,777,216 nodes, 277M edges with the
dangling repair and a planted hub of 1.57M out-edges), Zipf(1.5) weights in
[1, 1000], ~5 % dangling nodes, alpha = 0.15, R = 50, depth-3 segment tables
for out-degree <= 8, top-64 per source, Philox seed 1: the largest
single-GPU graph workload.  rmat20 (scale 20, alpha 0.2, R 100, top-32),
er1k, the 2048-instance batched workload and serving are the other lines.

Roofline of the walker: `frac` = DRAM bytes per launch (ncu, read + write,
per draw on a block-sampled capture of the same kernel source and launch
shape, times this launch's draws) / walker CUDA-event time / measured copy
peak.  Beside it, the 32-byte sectors the layout's searches read (counted
by a statistics launch) and the flat-CSR bisection model of the same draws.

--impl reference times the CPU oracle (single-threaded C) on a bounded sample
of the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import re
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat20": dict(alpha=0.2, R=100, seed=1, topk=32, segments=False,
                   desc="R-MAT scale 20, 16.8M edges (a=.57 b=.19 c=.19), Zipf(1.5) w in [1,1000], 5% dangling"),
    "er1k": dict(alpha=0.15, R=1000, seed=1, topk=32, segments=False,
                 desc="Erdos-Renyi n=1000 m=10000, w U[1,10], dense n x n counts"),
    "rmat24": dict(alpha=0.15, R=50, seed=1, topk=64, segments=True, launch=dict(refill_lanes=16, step_loads=6),
                   desc="R-MAT scale 24, 268M edges + hub > 1e6, Zipf(1.5) w in [1,1000], 5% dangling, "
                        "depth-3 segments for out-degree <= 8"),
    "rmat24plain": dict(alpha=0.15, R=50, seed=1, topk=64, segments=False, launch=dict(refill_lanes=16, step_loads=6),
                        desc="R-MAT scale 24 as rmat24, plain steps only"),
    "rmat20alias": dict(alpha=0.2, R=100, seed=1, topk=32, segments=False, sampler=1,
                        desc="R-MAT scale 20 as rmat20, integer alias sampler (Algorithm 1 tables built every step)"),
    "rmat24alias": dict(alpha=0.15, R=50, seed=1, topk=64, segments=False, sampler=1,
                        desc="R-MAT scale 24 as rmat24, integer alias sampler (Algorithm 1 tables built every step)"),
    "serve": dict(alpha=0.15, R=100, seed=1, topk=32, segments=False,
                  desc="queries on the R-MAT scale-24 graph resident on the device: |S| log-uniform in [1, 1e5] "
                       "distinct uniform sources, Poisson arrivals at rho x measured capacity"),
    "accuracy": dict(alpha=0.15, R=4096, seed=1, topk=1000, segments=False,
                     desc="Chung-Lu n=50000 (exponent 2.3, mean degree 12, w U[1,100]), 100 sources; NDCG/MAP@k of "
                          "the top-k rows against FP64 power iteration, R in {64, 256, 1024, 4096, 4x4096 tags}"),
    "sweep_alpha": dict(alpha=0.2, R=100, seed=1, topk=32, segments=False,
                        desc="rmat20 graph, alpha in {0.05, 0.1, 0.15, 0.2, 0.3, 0.5}: walker time and step rate"),
    "sweep_chunk": dict(alpha=0.2, R=100, seed=1, topk=32, segments=False,
                        desc="rmat20 graph, chunk_sources x warps_per_block grid against the autotuner's pick"),
    "chunglu2048alias": dict(alpha=0.15, R=200, seed=1, topk=32, segments=False, sampler=1,
                             desc="the 2048 Chung-Lu graphs of chunglu2048 with integer alias tables (built once, "
                                  "outside the replayed step)"),
    "chunglu2048": dict(alpha=0.15, R=200, seed=1, topk=32, segments=False,
                        desc="2048 Chung-Lu graphs (exponent 2.3, n log-uniform in [100, 50000], mean degree 12, "
                             "w U[1,100]) in one block-diagonal graph; one persistent launch replayed as a CUDA graph"),
}
L2_FLUSH_BYTES = 512 << 20


def base_graph(workload: str) -> str:
    """The graph a workload runs on (variants share their base graph)."""
    for suffix in ("plain", "alias"):
        workload = workload.replace(suffix, "")
    return workload


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_workload(n_src: int, rank: int, world: int):
    """Work of one rank: every source of its own replica of the graph, with the
    rank as the Philox tag, so each rank draws independent walks (summing the
    ranks' rows is the estimate with R * world walks per source).  Per-GPU work
    is fixed as the number of GPUs grows (weak scaling); no data moves between
    ranks."""
    return 0, n_src, rank


def reduce_over_ranks(seconds: float, units, world: int, dist=None, device=None):
    """Max of the timed seconds and sum of the processed units over ranks."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(x) for x in units], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(x) for x in u.tolist()]


def gc_pause():
    """Python's cyclic collector off over a timed region: a full collection of
    this process's objects takes tens of milliseconds and would land inside
    whichever step it interrupts (short steps are bound by host launches)."""
    gc.collect()
    gc.disable()


def gc_resume():
    gc.enable()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, path: str | None):
        self.path = path or os.path.join(tempfile.gettempdir(), f"ppr_clocks_{os.getpid()}.csv")
        self.device = device
        self.proc = None

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # nvidia-smi's start-up (NVML initialisation, some hundred ms of host
        # work) would otherwise overlap a short timed region whose steps are
        # bound by host launch latency: wait for its first sample (at most 3 s)
        t0 = time.perf_counter()
        while self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


RENUMBER = {"auto": None, "on": True, "off": False}  # --renumber -> ppr load_graph(renumber=...)


def _code_only(text: str) -> str:
    """Source text without comments and blank lines (a comment edit leaves the
    kernels, and so their recorded traffic, unchanged)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return "\n".join(ln for ln in lines if ln.strip())


def kernel_source_hash(root=None):
    """Hash of the walker's source files (the launch, the step, the layout and
    its build, the numbering), comments left out."""
    h = hashlib.sha256()
    for f in ("walk.cu", "walk_step.cuh", "ppr_internal.cuh", "renumber.cu", "graph.cu"):
        h.update(_code_only(open(os.path.join(root or ROOT, "paper_1903_11749_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, launch: dict, renumbered: bool = False):
    """The committed ncu DRAM figure of the walker (bytes per draw, read +
    write) for this workload, if it was taken on the current kernel source
    with the same launch shape and node numbering; else None."""
    p = os.path.join(ROOT, "profiles", "walker_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_source_hash():
        return None
    if e.get("launch", {}) != {k: v for k, v in launch.items() if v}:
        return None
    if bool(e.get("renumbered", False)) != bool(renumbered):
        return None
    return e


def sample_sources(n: int, every: int, block: int):
    """Profiling case: one block of `block` consecutive sources in every
    `every` blocks (block 1: every `every`-th source)."""
    if block <= 1:
        return np.arange(0, n, every, dtype=np.int32)
    starts = np.arange(0, n, block * every, dtype=np.int64)
    return np.concatenate([np.arange(s, min(n, s + block), dtype=np.int32) for s in starts])


def walker_roofline(workload, launch, sampled, draws, sectors, model_sectors, kernel_ms, peak, peak_kind,
                    renumbered=False):
    """Roofline of the walker launch.  frac is DRAM-based: the ncu DRAM
    bytes per draw recorded for this kernel source and launch shape, times
    the launch's draws, over the walker's CUDA-event time.  Without a current
    ncu record the counted layout sectors stand in and `basis` says so."""
    s = kernel_ms / 1e3
    counted = sectors * 32.0
    model = model_sectors * 32.0
    rec = None if sampled else recorded_traffic(workload, launch, renumbered)
    if rec is not None:
        traffic = rec["dram_bytes_per_draw"] * draws
        achieved, basis = traffic / s / 1e9, "ncu DRAM bytes (read + write) per draw x draws / walker time"
    else:
        traffic = None
        achieved, basis = counted / s / 1e9, "counted layout sectors / walker time (no current ncu DRAM record)"
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "basis": basis, "peak_kind": peak_kind, "kernel": "k_walk_persistent",
           "kernel_ms": kernel_ms, "draws": draws,
           "counted_sector_frac": counted / s / 1e9 / peak,
           "counted": {"bytes_per_launch": counted, "sectors_per_draw": sectors / max(draws, 1),
                       "model": "32-byte sectors the walker's own layout reads per draw: node record, one per "
                                "search-tree level below the record, 1-2 sectors of the bottom block (alias: "
                                "node record + slot), counted by a statistics launch"},
           "flat_csr_model": {"bytes_per_launch": model, "sectors_per_draw": model_sectors / max(draws, 1),
                              "frac": model / s / 1e9 / peak,
                              "model": "the same draws on a flat CSR searched by bisection without reuse: row_ptr "
                                       "sector + max(1, ceil(log2 d) - 1) probe sectors + col sector per draw"}}
    if rec is not None:
        out["traffic_record"] = {k: rec[k] for k in ("case", "dram_bytes_per_draw", "summary") if k in rec}
    return out


def host_cpu():
    """CPU model and logical core count of the host the oracle runs on."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model in ("", platform.machine()):
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"model": model, "machine": platform.machine(), "nproc": os.cpu_count()}


def cpu_baseline(g, wl, budget_s: float = 15.0):
    """The oracle as it stands (single-threaded C + numpy counting) on an evenly
    strided sample of sources; returns steps/s and a description."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    O.build()
    og = O.prepare(g.n, g.row_ptr, g.col, g.w)
    # calibrate on a small sample, then size the sample to the budget
    t0 = time.perf_counter()
    seg = dict(segments=wl["segments"], lazy_segments=True, sampler=wl.get("sampler", 0))
    ends, steps = O.walks(og, wl["alpha"], wl["R"], wl["seed"], 0, 200, **seg)
    dt = max(time.perf_counter() - t0, 1e-3)
    n_src = int(max(200, min(g.n, 200 * budget_s / dt)))
    stride = max(1, g.n // n_src)
    total_steps, total_walks, t_all = 0, 0, 0.0
    srcs = range(0, g.n, stride)
    t0 = time.perf_counter()
    # contiguous blocks of 64 sources, strided over the whole id range
    for s in list(srcs)[: max(1, n_src // 64)]:
        e, st = O.walks(og, wl["alpha"], wl["R"], wl["seed"], s, min(g.n, s + 64), **seg)
        rp, col, cnt = O.rows(e, g.n)
        if wl["topk"]:
            O.topk(rp, col, cnt, wl["topk"])
        total_steps += st
        total_walks += e.size
    t_all = time.perf_counter() - t0
    return {"value": total_steps / t_all, "unit": "walk steps/s", "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "walks_per_s": total_walks / t_all,
            "sample": f"{total_walks // wl['R']} sources in blocks of 64 strided over all {g.n} sources, "
                      f"{total_walks} walks, {total_steps} steps, {t_all:.1f} s"}


def run_reference_batched(args, wl, I, O):
    """Oracle on a bounded sample of the batched workload: the first 64
    sources of every 128th instance, each instance walked with its id as tag."""
    inst = I.chung_lu_instances(2048, 100, 50_000, 12.0, 2.3, 1, 100, seed=4242)
    subs = [(gi, inst.instance(gi)) for gi in range(0, inst.count, 128)]
    ogs = [(gi, O.prepare(sg.n, sg.row_ptr, sg.col, sg.w), sg.n) for gi, sg in subs]
    per_step, st_tot, wk_tot = [], 0, 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st = wk = 0
        for gi, og, n in ogs:
            e, stp = O.walks(og, wl["alpha"], wl["R"], wl["seed"], 0, min(n, 64), tag=gi,
                             sampler=wl.get("sampler", 0))
            rp, c, cn = O.rows(e, n)
            O.topk(rp, c, cn, wl["topk"])
            st += stp
            wk += e.size
        if it >= args.warmup:
            per_step.append(time.perf_counter() - t0)
            st_tot += st
            wk_tot += wk
    T = sum(per_step)
    sample = f"first 64 sources of every 128th instance ({len(ogs)} instances) per step"
    line = {"impl": "reference", "metric": "walk steps/s", "value": st_tot / T, "unit": "walk steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "alpha": wl["alpha"], "R": wl["R"],
                       "topk": wl["topk"]},
            "walks_per_s": wk_tot / T,
            "cpu_baseline": {"value": st_tot / T, "unit": "walk steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": st_tot / T, "unit": "walk steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_1903_11749_gb300 import inputs as I
    wl = WORKLOADS[args.workload]
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    O.build()
    if args.workload.startswith("chunglu2048"):
        return run_reference_batched(args, wl, I, O)
    if args.workload in ("serve", "accuracy") or args.workload.startswith("sweep_"):
        print(json.dumps({"impl": "reference", "unavailable": f"the {args.workload} workload has no oracle arm; "
                          "its graph workloads (rmat24, rmat20) do"}))
        return 0
    g = I.workload_graph(base_graph(args.workload))
    og = O.prepare(g.n, g.row_ptr, g.col, g.w)
    n_blk = 64
    per_step = []
    steps_tot = walks_tot = 0
    rng_src = np.linspace(0, g.n - n_blk, num=max(1, args.ref_blocks), dtype=np.int64)
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st_step, wk = 0, 0
        for s in rng_src:
            e, st = O.walks(og, wl["alpha"], wl["R"], wl["seed"], int(s), int(s) + n_blk,
                            segments=wl["segments"], lazy_segments=True, sampler=wl.get("sampler", 0))
            rp, col, cnt = O.rows(e, g.n)
            O.topk(rp, col, cnt, wl["topk"])
            st_step += st
            wk += e.size
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            per_step.append(dt)
            steps_tot += st_step
            walks_tot += wk
    T = sum(per_step)
    val = steps_tot / T
    sample = f"{len(rng_src) * n_blk} sources per step ({len(rng_src)} blocks of {n_blk} spread over {g.n})"
    line = {"impl": "reference", "metric": "walk steps/s", "value": val, "unit": "walk steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "alpha": wl["alpha"], "R": wl["R"],
                       "topk": wl["topk"], "sources_per_step": len(rng_src) * n_blk},
            "walks_per_s": walks_tot / T,
            "cpu_baseline": {"value": val, "unit": "walk steps/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "walk steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(args):
    """Many small graphs in one fused persistent launch, recorded once as a
    CUDA graph (ppr_run_into: caller workspace, no allocation) and replayed
    every step; launch tuning from the autotuner (cached as JSON)."""
    import torch
    from paper_1903_11749_gb300 import build as B
    from paper_1903_11749_gb300 import inputs as I
    from paper_1903_11749_gb300 import tune
    B.build()
    from paper_1903_11749_gb300 import ppr
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    else:
        dist = None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    inst = I.chung_lu_instances(2048, 100, 50_000, 12.0, 2.3, 1, 100, seed=4242)
    N = int(inst.node_off[-1])
    ctx = ppr.Context(local)
    G = ctx.load_graph_batch(inst.node_off, inst.row_ptr, inst.col, inst.w)
    run_kw = dict(alpha=wl["alpha"], R=wl["R"], seed=wl["seed"], topk=wl["topk"], sampler=wl.get("sampler", 0))
    t0 = time.perf_counter()
    tun = tune.tuned(G, torch.cuda.get_device_name(dev), sample_sources=400_000, **run_kw)
    tune_s = time.perf_counter() - t0
    lk = tune.launch_kwargs(tun)
    # statistics pass: draws and algorithmic sectors of one full pass
    r = G.run(stats=True, **run_kw, **lk)
    info = r.info()
    draws, sectors, walks = int(info.steps), int(info.sectors), int(info.walks)
    model_sectors = int(info.model_sectors)
    del r
    # walker-only time (for the roofline) from an eager run
    kms = []
    for _ in range(2):
        r = G.run(**run_kw, **lk)
        kms.append(r.info().kernel_ms)
        del r
    cap = min(wl["R"], int(np.diff(inst.node_off).max()))
    k = wl["topk"]
    ws = torch.empty(G.workspace_size(**run_kw, **lk), dtype=torch.uint8, device=dev)
    nnz = torch.empty(N, dtype=torch.int32, device=dev)
    cols = torch.empty(N * cap, dtype=torch.int32, device=dev)
    cnts = torch.empty(N * cap, dtype=torch.int32, device=dev)
    ti = torch.empty((N, k), dtype=torch.int32, device=dev)
    tc = torch.empty((N, k), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, tag=0, **run_kw, **lk)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        G.run_into(ws, nnz, cols, cnts, cap, ti, tc, stream=s, tag=0, **run_kw, **lk)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local, None)
    clocks.start()
    launches0 = ppr.kernel_launches()
    step_ms = []
    gc_pause()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        cs = torch.cuda.current_stream(dev)
        e0.record(cs)
        graph.replay()
        e1.record(cs)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize(dev)
    gc_resume()
    clk = clocks.stop()
    T_max, units = reduce_over_ranks(sum(step_ms) / 1e3, [draws * args.steps, walks * args.steps], world, dist, dev)
    # kernels per replay: chunk count, 3 scan kernels, chunk fill, walker, reduction
    launches = 7 * args.steps
    # the unfused alternatives on the same GB300
    r = G.run(kernel=ppr.KERNEL_PLAIN, **run_kw)
    r = G.run(kernel=ppr.KERNEL_PLAIN, **run_kw)
    plain_ms = r.info().run_ms
    del r
    t0 = time.perf_counter()
    per_inst_ms = 0.0
    for gi in range(inst.count):
        r = G.run(src_begin=int(inst.node_off[gi]), src_end=int(inst.node_off[gi + 1]), **run_kw, **lk)
        per_inst_ms += r.info().run_ms
        del r
    per_inst_wall = time.perf_counter() - t0
    peak, peak_kind = measured_peaks()
    kms_ = statistics.mean(kms)
    roofline = walker_roofline(args.workload, lk, False, draws, sectors, model_sectors, kms_, peak, peak_kind)
    # end to end: host CSR in (pinned), one run, rows + top-k out (pinned)
    e2e = None
    if not args.no_e2e:
        h = [torch.from_numpy(x).pin_memory() for x in (inst.row_ptr, inst.col, inst.w.view(np.int32))]
        o_rp = torch.empty(N + 1, dtype=torch.int64).pin_memory()
        o_col = torch.empty(N * cap, dtype=torch.int32).pin_memory()
        o_cnt = torch.empty(N * cap, dtype=torch.int32).pin_memory()
        o_ti = torch.empty((N, k), dtype=torch.int32).pin_memory()
        o_tc = torch.empty((N, k), dtype=torch.int32).pin_memory()
        times = []
        gc_pause()
        for it in range(3):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            Gh = ctx.load_graph_batch(inst.node_off, h[0], h[1], h[2])
            r = Gh.run(**run_kw, **lk)
            nz = r.sparse_rows_into(o_rp, o_col, o_cnt)
            r.topk_into(k, o_ti, o_tc)
            if it > 0:
                times.append(time.perf_counter() - t0)
            del r, Gh
        gc_resume()
        e2e = {"value": draws / statistics.mean(times), "unit": "walk steps/s",
               "h2d_bytes_per_step": int(inst.row_ptr.nbytes + inst.col.nbytes + inst.w.nbytes),
               "d2h_bytes_per_step": int((N + 1) * 8 + nz * 8 + N * k * 8), "ms_per_step": 1e3 * statistics.mean(times)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sys.path.insert(0, os.path.join(ROOT, "oracle"))
        import oracle as O
        O.build()
        st = wk = 0
        t0 = time.perf_counter()
        for gi in range(0, inst.count, 128):
            sub = inst.instance(gi)
            og = O.prepare(sub.n, sub.row_ptr, sub.col, sub.w)
            e, stp = O.walks(og, wl["alpha"], wl["R"], wl["seed"], 0, min(sub.n, 64), tag=gi,
                             sampler=wl.get("sampler", 0))
            rp_, c_, n_ = O.rows(e, sub.n)
            O.topk(rp_, c_, n_, k)
            st += stp
            wk += e.size
        dt = time.perf_counter() - t0
        cpu = {"value": st / dt, "unit": "walk steps/s", "cores": 1, "kind": "oracle", "walks_per_s": wk / dt,
               "sample": f"first 64 sources of every 128th instance ({inst.count // 128} instances), {wk} walks, "
                         f"{st} steps, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": "walk steps/s", "value": units[0] / T_max, "unit": "walk steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": args.workload, "desc": wl["desc"], "alpha": wl["alpha"], "R": wl["R"],
                           "topk": k, "instances": inst.count, "n": N, "m": int(inst.row_ptr[-1]),
                           "parallelism": "1 GPU", "l2": "flushed between steps (512 MB write)",
                           "step": "one CUDA-graph replay: chunk table, fused persistent walker, reduction",
                           "tuning": tun, "tune_seconds": tune_s},
                "walks_per_s": units[1] / T_max, "steps_per_walk": draws / max(walks, 1),
                "roofline": roofline,
                "plain_kernel": {"value": draws / (plain_ms / 1e3), "unit": "walk steps/s", "ms_per_step": plain_ms,
                                 "kernel": "one thread per walk over all instances + reduction"},
                "unfused_per_instance": {"value": draws / (per_inst_ms / 1e3), "unit": "walk steps/s",
                                         "device_ms": per_inst_ms, "wall_s": per_inst_wall,
                                         "kernel": "one persistent run per instance (2048 runs)"},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """Continuous-batching service on the scale-24 graph: first the capacity
    (queries submitted back to back), then a Poisson stream at rho x that rate;
    latency = completion - submission (steady clock, inside the library)."""
    import threading
    import torch
    from paper_1903_11749_gb300 import build as B
    from paper_1903_11749_gb300 import inputs as I
    B.build()
    from paper_1903_11749_gb300 import ppr
    rank, world, local = env_rank()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    wl = WORKLOADS["serve"]
    g = I.workload_graph("rmat24")
    ctx = ppr.Context(local)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w, renumber=RENUMBER[args.renumber])
    rng = np.random.Generator(np.random.PCG64(777))
    smax = 100_000
    n_warm, n_meas = args.serve_warmup, args.serve_queries

    def make_queries(k):
        sizes = np.floor(np.exp(rng.uniform(0.0, np.log(smax), k))).astype(np.int64)
        return [rng.choice(g.n, size=int(s), replace=False).astype(np.int32) for s in sizes]

    kw = dict(alpha=wl["alpha"], R=wl["R"], seed=wl["seed"], topk=wl["topk"])
    # the launch shape of the scale-24 workload of the same sampler
    launch = WORKLOADS["rmat24plain" if args.serve_sampler == 0 else "rmat24alias"].get("launch", {})
    launch = {k: v for k, v in launch.items() if k in ("refill_lanes", "chunk_sources")}

    def run_stream(queries, rate):
        """Submit at Poisson times (rate queries/s; 0 = back to back), poll all."""
        ids = [None] * len(queries)
        gaps = rng.exponential(1.0 / rate, len(queries)) if rate > 0 else np.zeros(len(queries))
        t_start = time.perf_counter()

        def submitter():
            t_next = t_start
            for i, q in enumerate(queries):
                t_next += gaps[i]
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                ids[i] = ctx.submit(q, **kw)

        th = threading.Thread(target=submitter)
        th.start()
        stats = []
        for i, q in enumerate(queries):
            while ids[i] is None:
                time.sleep(0.0002)
            stats.append(ctx.poll(ids[i], len(q), kw["topk"], timeout_ms=600000)[2])
        th.join()
        return stats

    def measure(mode):
        """Capacity (queries back to back), then a Poisson stream at each rho."""
        ctx.serve_start(G, streams=args.serve_streams, max_sources=smax, max_topk=wl["topk"],
                        sampler=args.serve_sampler, mode=mode, **launch)
        warm = make_queries(n_warm)
        st = run_stream(warm, 0)  # back to back: the service capacity
        t0 = min(x["submit_ns"] for x in st)
        t1 = max(x["done_ns"] for x in st)
        cap_walks = sum(x["walks"] for x in st) / ((t1 - t0) / 1e9)
        results = {}
        clocks = Clocks(local, None)
        clocks.start()
        launches0 = ppr.kernel_launches()
        for rho in args.serve_rho:
            qs = make_queries(n_meas)
            rate = rho * cap_walks / (((smax - 1) / np.log(smax)) * wl["R"])
            st = run_stream(qs, rate)
            lat = np.array([(x["done_ns"] - x["submit_ns"]) / 1e6 for x in st])
            t0 = min(x["submit_ns"] for x in st)
            t1 = max(x["done_ns"] for x in st)
            walks = sum(x["walks"] for x in st)
            small = np.array([x["sources"] <= 100 for x in st])
            results[str(rho)] = {"queries": len(qs), "rate_qps": rate, "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                                 "p99_ms_small_queries": float(np.percentile(lat[small], 99)) if small.any() else None,
                                 "walks_per_s": walks / ((t1 - t0) / 1e9), "seconds": (t1 - t0) / 1e9}
        clk = clocks.stop()
        launches = ppr.kernel_launches() - launches0  # every measured stream (all rho)
        info = ctx.serve_info()
        ctx.serve_stop()
        return {"capacity_walks_per_s": cap_walks, "by_rho": results, "clocks": clk, "gpu_launches": launches,
                "loop_launches": info["launches"] if mode == ppr.SERVE_DEVICE_LOOP else None,
                "loop_activity": ({k: info[k] for k in ("draws", "iterations", "claims", "claim_misses", "sleeps",
                                                         "reduced", "idle_exits", "cycles_claim", "cycles_step",
                                                         "cycles_sleep", "cycles_total", "grid_blocks")}
                                  if mode == ppr.SERVE_DEVICE_LOOP else None)}

    mode = ppr.SERVE_STREAMS if args.serve_mode == "streams" else ppr.SERVE_DEVICE_LOOP
    res = measure(mode)
    other = None
    if args.serve_compare:
        other = measure(ppr.SERVE_DEVICE_LOOP if mode == ppr.SERVE_STREAMS else ppr.SERVE_STREAMS)
    T = ppr.alpha_threshold(wl["alpha"])
    main_r = res["by_rho"][str(args.serve_rho[0])]
    mean_walks = (((smax - 1) / np.log(smax))) * wl["R"]
    line = {"metric": "walk steps/s", "value": main_r["walks_per_s"] * (2.0 ** 32 / T), "unit": "walk steps/s",
            "n_gpus": 1, "steps": n_meas, "warmup": n_warm, "ms_per_step": main_r["mean_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "serve", "desc": wl["desc"], "alpha": wl["alpha"], "R": wl["R"], "topk": wl["topk"],
                       "n": g.n, "m": g.m, "mode": args.serve_mode,
                       "streams": args.serve_streams if mode == ppr.SERVE_STREAMS else None,
                       "sampler": "alias" if args.serve_sampler == 1 else "prefix", "launch": launch,
                       "steps_counted": "expected steps walks*2^32/T of the delivered walks",
                       "step": "one query (ms_per_step = mean latency, submit to completion)"},
            "p50_ms": main_r["p50_ms"], "p99_ms": main_r["p99_ms"], "walks_per_s": main_r["walks_per_s"],
            "capacity_walks_per_s": res["capacity_walks_per_s"], "mean_walks_per_query": mean_walks,
            "by_rho": res["by_rho"], "loop_launches": res["loop_launches"], "loop_activity": res["loop_activity"],
            "other_mode": ({"mode": "streams" if mode == ppr.SERVE_DEVICE_LOOP else "device_loop",
                            "capacity_walks_per_s": other["capacity_walks_per_s"], "by_rho": other["by_rho"]}
                           if other else None),
            "clocks": res["clocks"], "gpu_launches": res["gpu_launches"]}
    print(json.dumps(line))
    return 0


def run_accuracy(args):
    """Accuracy analog of the paper's NDCG/MAP experiment (Sec. 5.2): top-k
    rows of the CUDA path against the exact ranking from FP64 power
    iteration, for growing R, plus Definition 1 at the walk count of
    ppr_walks_for_accuracy (eps 0.5, p_f 0.01)."""
    import torch
    from paper_1903_11749_gb300 import accuracy as A
    from paper_1903_11749_gb300 import build as B
    from paper_1903_11749_gb300 import inputs as I
    B.build()
    from paper_1903_11749_gb300 import ppr
    rank, world, local = env_rank()
    if rank != 0:
        return 0
    wl = WORKLOADS["accuracy"]
    g = I.chung_lu_graph(50_000, avg_deg=12.0, exponent=2.3, wlo=1, whi=100, seed=5050)
    src = np.linspace(0, g.n - 1, 100).astype(np.int32)
    T = ppr.alpha_threshold(wl["alpha"])
    t0 = time.perf_counter()
    pi = A.exact_ppr_rows(g.n, g.row_ptr, g.col, g.w, src, T, tol=1e-12)
    truth_s = time.perf_counter() - t0
    ctx = ppr.Context(local)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    ks = (10, 100, 1000)
    eps, p_f = 0.5, 0.01
    table = []
    for R, runs in ((64, 1), (256, 1), (1024, 1), (4096, 1), (4096, 4)):
        est = np.zeros((len(src), g.n))
        idx = cnt = None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for tag in range(runs):
            res = G.run_list(src, alpha=wl["alpha"], R=R, seed=wl["seed"], tag=tag, topk=max(ks))
            rp, col, c = res.sparse_rows()
            np.add.at(est, (np.repeat(np.arange(len(src)), np.diff(rp)), col), c)
            if runs == 1:
                idx, cnt = res.topk()
        e1.record()
        e1.synchronize()
        est /= R * runs
        row = {"R": R * runs, "runs": runs, "gpu_ms": e0.elapsed_time(e1)}
        for k in ks:
            nd, ap = [], []
            for i in range(len(src)):
                truth = A.exact_topk(pi[i], k)
                if runs == 1:
                    pred = A.estimated_ranking(idx[i], cnt[i])
                else:
                    pred = A.exact_topk(est[i], k)  # same order rule on the summed counts
                nd.append(A.ndcg_at_k(pred, truth, k))
                ap.append(A.average_precision_at_k(pred, truth, k))
            row[f"ndcg@{k}"] = float(np.mean(nd))
            row[f"map@{k}"] = float(np.mean(ap))
        delta = A.delta_for_walks(R * runs, eps, p_f)
        bad, pairs = A.definition1_violations(est, pi, eps, delta)
        row.update({"def1_delta": delta, "def1_pairs": pairs, "def1_violations": bad})
        table.append(row)
    last = table[3]
    line = {"metric": "NDCG@100", "value": last["ndcg@100"], "unit": "ratio", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "accuracy", "desc": wl["desc"], "alpha": wl["alpha"], "n": g.n, "m": g.m,
                       "sources": len(src), "eps": eps, "p_f": p_f},
            "truth": f"FP64 power iteration to active mass < 1e-12 ({truth_s:.1f} s on the host)",
            "table": table}
    print(json.dumps(line))
    return 0


def run_sweep(args):
    """Parameter sweeps on the rmat20 graph (analogs of the paper's gamma and
    alpha experiments, Sec. 5.3-5.4): for each setting, the mean of --steps
    runs after --warmup, walker time from the library's events and the whole
    run (walks + reduction) from events on the stream."""
    import torch
    from paper_1903_11749_gb300 import build as B
    from paper_1903_11749_gb300 import inputs as I
    B.build()
    from paper_1903_11749_gb300 import ppr
    rank, world, local = env_rank()
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    g = I.workload_graph("rmat20")
    ctx = ppr.Context(local)
    G = ctx.load_graph(g.n, g.row_ptr, g.col, g.w)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(**kw):
        for _ in range(args.warmup):
            G.run(stream=stream, **kw)
        walk, whole, steps = [], [], 0
        for _ in range(max(1, args.steps)):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = G.run(stream=stream, wait=False, **kw)
            e1.record(stream)
            r.wait()
            e1.synchronize()
            whole.append(e0.elapsed_time(e1))
            walk.append(r.info().kernel_ms)
            steps = int(r.info().steps)
        ms = statistics.mean(whole)
        return {"walker_ms": statistics.mean(walk), "run_ms": ms, "steps": steps,
                "steps_per_s": steps / (ms / 1e3)}

    base = dict(R=wl["R"], seed=wl["seed"], topk=wl["topk"])
    table = []
    if args.workload == "sweep_alpha":
        for alpha in (0.05, 0.1, 0.15, 0.2, 0.3, 0.5):
            row = {"alpha": alpha}
            row.update(timed(alpha=alpha, **base))
            table.append(row)
        best = max(table, key=lambda r: r["steps_per_s"])
        metric, value, unit = "walk steps/s at alpha 0.2", next(r for r in table if r["alpha"] == 0.2)["steps_per_s"], \
            "walk steps/s"
    else:
        for wpb in (4, 8):
            for cs in (1, 2, 4, 8, 16, 32):
                row = {"warps_per_block": wpb, "chunk_sources": cs}
                row.update(timed(alpha=wl["alpha"], warps_per_block=wpb, chunk_sources=cs, **base))
                table.append(row)
        t = G.autotune(sample_sources=200_000, alpha=wl["alpha"], **base)
        pick = {"warps_per_block": t["warps_per_block"], "chunk_sources": t["chunk_sources"],
                "large_degree": t["large_degree"], "refill_lanes": t["refill_lanes"], "autotuner": True}
        pick.update(timed(alpha=wl["alpha"], warps_per_block=t["warps_per_block"], chunk_sources=t["chunk_sources"],
                          large_degree=t["large_degree"], refill_lanes=t["refill_lanes"], **base))
        table.append(pick)
        best = max(table[:-1], key=lambda r: r["steps_per_s"])
        metric, value, unit = "autotuned / best grid point", pick["steps_per_s"] / best["steps_per_s"], "ratio"
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "R": wl["R"], "topk": wl["topk"],
                       "n": g.n, "m": g.m, "l2": "flushed before every run (512 MB write)"},
            "best": best, "table": table}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--ref-blocks", type=int, default=48)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--warps-per-block", type=int, default=0)
    ap.add_argument("--chunk-sources", type=int, default=0)
    ap.add_argument("--large-degree", type=int, default=0)
    ap.add_argument("--refill-lanes", type=int, default=0,
                    help="persistent walker: idle lanes before a warp starts new walks (0 = 1)")
    ap.add_argument("--step-loads", type=int, default=0,
                    help="persistent walker: dependent loads per lane per warp iteration (0 = library default, -1 = "
                         "no bound)")
    ap.add_argument("--tune", action="store_true",
                    help="graph workloads: launch shape from the autotuner (cached) instead of the workload's")
    ap.add_argument("--l2-persist", type=int, default=0, choices=[0, 1],
                    help="walker launches keep the node records persisting in L2")
    ap.add_argument("--renumber", default="auto", choices=["auto", "on", "off"],
                    help="layout node numbering: by in-degree (on), the generator's (off), or the library's choice")
    ap.add_argument("--serve-queries", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-rho", type=float, nargs="+", default=[0.5, 0.8])
    ap.add_argument("--serve-sampler", type=int, default=0, choices=[0, 1],
                    help="neighbour choice of the served queries (1: integer alias tables)")
    ap.add_argument("--serve-mode", default="device_loop", choices=["device_loop", "streams"],
                    help="serving: the resident device loop, or one launch per query on a few streams")
    ap.add_argument("--serve-compare", action="store_true",
                    help="serving: also measure the other mode on the same queries' distribution")
    ap.add_argument("--sample-every", type=int, default=0,
                    help="profiling case: walk only one source (or block of sources) in every k (an explicit list)")
    ap.add_argument("--sample-block", type=int, default=1,
                    help="profiling case: consecutive sources per sampled block")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("chunglu2048"):
        return run_batched(args)
    if args.workload == "serve":
        return run_serving(args)
    if args.workload == "accuracy":
        return run_accuracy(args)
    if args.workload.startswith("sweep_"):
        return run_sweep(args)

    import torch
    import torch.distributed as dist
    from paper_1903_11749_gb300 import build as B
    from paper_1903_11749_gb300 import inputs as I
    B.build()
    from paper_1903_11749_gb300 import ppr

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    renum = RENUMBER[args.renumber]
    g = I.workload_graph(base_graph(args.workload))
    a, b, rank_tag = rank_workload(g.n, rank, world)
    tune = dict(warps_per_block=args.warps_per_block, chunk_sources=args.chunk_sources,
                large_degree=args.large_degree, l2_persist=args.l2_persist, refill_lanes=args.refill_lanes,
                step_loads=args.step_loads)

    ctx = ppr.Context(local)
    stream = torch.cuda.current_stream(dev)
    d_rp = torch.from_numpy(g.row_ptr).to(dev)
    d_col = torch.from_numpy(g.col).to(dev)
    d_w = torch.from_numpy(g.w.view(np.int32)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    # launch shape: the workload's (picked offline by the autotuner and the
    # refill sweep), or the command line's, or the autotuner's now (--tune);
    # tuning never changes results
    tuning = None
    if not any((args.warps_per_block, args.chunk_sources, args.large_degree, args.refill_lanes, args.step_loads)):
        tune.update(wl.get("launch", {}))
    if args.tune:
        from paper_1903_11749_gb300 import tune as tuner
        Gt = ctx.load_graph(g.n, d_rp, d_col, d_w, stream=stream, m=g.m, renumber=renum)
        t0 = time.perf_counter()
        tuning = tuner.tuned(Gt, torch.cuda.get_device_name(dev), sample_sources=400_000, alpha=wl["alpha"], R=wl["R"],
                             seed=wl["seed"], topk=wl["topk"], segments=wl["segments"], sampler=wl.get("sampler", 0))
        tuning = dict(tuning, seconds=time.perf_counter() - t0)
        tune.update(tuner.launch_kwargs(tuning))
        del Gt

    sample = sample_sources(b, args.sample_every, args.sample_block) if args.sample_every > 0 else None

    def step(kernel=ppr.KERNEL_PERSISTENT, stats=False):
        G = ctx.load_graph(g.n, d_rp, d_col, d_w, stream=stream, m=g.m, renumber=renum)
        kw = dict(alpha=wl["alpha"], R=wl["R"], seed=wl["seed"], tag=rank_tag, topk=wl["topk"],
                  segments=wl["segments"], kernel=kernel, stats=stats, stream=stream, wait=False,
                  sampler=wl.get("sampler", 0), **tune)
        if sample is not None:
            r = G.run_list(sample, **kw)
        else:
            r = G.run(src_begin=a, src_end=b, **kw)
        return G, r

    # statistics launch (untimed): exact draws and algorithmic sectors of one pass
    G0, r0 = step(stats=True)
    r0.wait()
    info0 = r0.info()
    draws_per_pass, sectors_per_pass, walks_per_pass = int(info0.steps), int(info0.sectors), int(info0.walks)
    model_per_pass = int(info0.model_sectors)
    renumbered = bool(G0.info().renumbered)
    # walk steps of one pass: the counted steps; with segment tables one draw
    # stands for up to three steps, so the plain-equivalent count walks * 2^32/T
    # (the expected number of steps) is used instead
    T_int = ppr.alpha_threshold(wl["alpha"])
    steps_per_pass = walks_per_pass * (2.0 ** 32 / T_int) if wl["segments"] else draws_per_pass
    del r0, G0

    for _ in range(args.warmup):
        G, r = step()
        r.wait()
        del r, G  # freed here, not inside the first timed step
    kernel_ms = []
    run_ms = []
    step_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local, None)
    clocks.start()
    launches0 = ppr.kernel_launches()
    gc_pause()
    for _ in range(args.steps):
        flush.fill_(1)  # L2 flush outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G, r = step()
        e1.record(stream)
        r.wait()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kernel_ms.append(r.info().kernel_ms)
        run_ms.append(r.info().run_ms)
        del r, G
    torch.cuda.synchronize(dev)
    gc_resume()
    launches = ppr.kernel_launches() - launches0
    clk = clocks.stop()
    T = sum(step_ms) / 1e3
    T_max, units = reduce_over_ranks(T, [steps_per_pass * args.steps, walks_per_pass * args.steps], world, dist, dev)
    value = units[0] / T_max
    walks_s = units[1] / T_max

    # plain one-thread-per-walk kernel on the same pass, for comparison
    # (short steps: as many warm-up and timed steps as the persistent kernel,
    # under a clock sampler of its own, so both see the same host conditions)
    plain = None
    if not args.no_plain:
        short = bool(step_ms) and statistics.mean(step_ms) < 10
        for _ in range(max(1, args.warmup if short else 1)):
            G, r = step(kernel=ppr.KERNEL_PLAIN)
            r.wait()
            del r, G
        pm, pk = [], []
        pclocks = Clocks(local, None)
        pclocks.start()
        gc_pause()
        for _ in range(max(1, args.steps if short else min(3, args.steps))):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G, r = step(kernel=ppr.KERNEL_PLAIN)
            e1.record(stream)
            r.wait()
            e1.synchronize()
            pm.append(e0.elapsed_time(e1))
            pk.append(r.info().kernel_ms)
            del r, G
        gc_resume()
        pclk = pclocks.stop()
        plain = {"value": steps_per_pass / (statistics.mean(pm) / 1e3), "unit": "walk steps/s",
                 "kernel_ms": statistics.mean(pk), "steps": len(pm),
                 "ms_per_step": statistics.mean(pm), "kernel": "one thread per walk + separate aggregation",
                 "clocks": pclk}

    # end to end through the C ABI with host buffers: pinned CSR in, rows + top-k out to pinned memory
    e2e = None
    if not args.no_e2e:
        h_rp = torch.from_numpy(g.row_ptr).pin_memory()
        h_col = torch.from_numpy(g.col).pin_memory()
        h_w = torch.from_numpy(g.w.view(np.int32)).pin_memory()
        h2d = g.row_ptr.nbytes + g.col.nbytes + g.w.nbytes
        S = b - a
        cap_rows = S * min(wl["R"], g.n)
        o_rp = torch.empty(S + 1, dtype=torch.int64).pin_memory()
        o_col = torch.empty(cap_rows, dtype=torch.int32).pin_memory()
        o_cnt = torch.empty(cap_rows, dtype=torch.int32).pin_memory()
        k = max(1, wl["topk"])
        o_ti = torch.empty((S, k), dtype=torch.int32).pin_memory()
        o_tc = torch.empty((S, k), dtype=torch.int32).pin_memory()
        run_kw = dict(alpha=wl["alpha"], R=wl["R"], seed=wl["seed"], src_begin=a, src_end=b, tag=rank_tag,
                      topk=wl["topk"], segments=wl["segments"], stream=stream, sampler=wl.get("sampler", 0), **tune)
        ti_arg = (o_ti, o_tc) if wl["topk"] else (None, None)

        load_call_ms = []  # host time until ppr_load_graph returns (its copies and build run on)

        def e2e_once(pipelined):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            G = ctx.load_graph(g.n, h_rp, h_col, h_w, stream=stream, m=g.m, renumber=renum)
            if pipelined:
                load_call_ms.append(1e3 * (time.perf_counter() - t0))
            if pipelined:  # rows and top-k copied to the host batch by batch, behind the walks
                nnz, _ = G.run_to_host(o_rp, o_col, o_cnt, *ti_arg, **run_kw)
            else:  # run, then read everything back
                r = G.run(**run_kw)
                nnz = r.sparse_rows_into(o_rp, o_col, o_cnt)
                if wl["topk"]:
                    r.topk_into(wl["topk"], o_ti, o_tc)
                del r
            t1 = time.perf_counter()
            del G
            return t1 - t0, nnz

        times, serial_times, nnz = [], [], 0
        gc_pause()
        for it in range(1 + min(5, args.steps)):
            dt, nnz = e2e_once(True)
            if it > 0:
                times.append(dt)
        for it in range(1 + min(2, args.steps)):
            dt, _ = e2e_once(False)
            if it > 0:
                serial_times.append(dt)
        gc_resume()
        d2h = o_rp.numel() * 8 + nnz * 8 + (S * wl["topk"] * 8 if wl["topk"] else 0)
        # the median iteration: host-timed iterations catch occasional host stalls
        e2e = {"value": steps_per_pass / statistics.median(times), "unit": "walk steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * statistics.median(times),
               "ms_mean": 1e3 * statistics.mean(times), "ms_each": [1e3 * t for t in times],
               "load_call_ms_each": load_call_ms[1:],
               "call": "ppr_load_graph (pinned host CSR) + ppr_run_to_host (pinned host rows and top-k)",
               "unpipelined": {"value": steps_per_pass / statistics.median(serial_times),
                               "ms_per_step": 1e3 * statistics.median(serial_times),
                               "call": "ppr_load_graph + ppr_run + ppr_sparse_rows + ppr_topk"}}

    peak, peak_kind = measured_peaks()
    kms = statistics.mean(kernel_ms)
    roofline = walker_roofline(args.workload, tune, sample is not None, draws_per_pass, sectors_per_pass,
                               model_per_pass, kms, peak, peak_kind, renumbered)
    roofline["walk_and_reduce_ms"] = statistics.mean(run_ms)

    # practical ceilings: dependent random 32-byte sector reads over a buffer
    # the size of the walked layout, and Philox draws with no memory traffic
    G = ctx.load_graph(g.n, d_rp, d_col, d_w, stream=stream, m=g.m, renumber=renum)
    if wl.get("sampler", 0) == 1:
        G.run(alpha=wl["alpha"], R=1, seed=1, src_begin=0, src_end=1, sampler=1, stream=stream)  # alias tables
    footprint = max(int(G.info().device_bytes), 64 << 20)
    del G
    chains_s, _ = ctx.probe_rate(0, footprint)
    gather_s, _ = ctx.probe_rate(2, footprint)
    philox_s, _ = ctx.probe_rate(1)
    walker_sectors_s = sectors_per_pass / (kms / 1e3)
    probe = {"buffer_bytes": footprint,
             "gather_sectors_per_s": gather_s, "gather_gbs": gather_s * 32 / 1e9,
             "chains_sectors_per_s": chains_s, "chains_gbs": chains_s * 32 / 1e9,
             "philox_draws_per_s": philox_s, "walker_sectors_per_s": walker_sectors_s,
             "walker_frac_of_gather": walker_sectors_s / gather_s,
             "walker_draws_per_s_over_philox": (draws_per_pass / (kms / 1e3)) / philox_s,
             "note": "uniform addresses over a buffer the size of the graph layout; the walks revisit hot nodes"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, wl, args.cpu_budget)

    if rank == 0:
        line = {"metric": "walk steps/s", "value": value, "unit": "walk steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": args.workload, "desc": wl["desc"], "alpha": wl["alpha"], "R": wl["R"],
                           "topk": wl["topk"], "n": g.n, "m": g.m, "sources": g.n,
                           "parallelism": f"{world} independent replicas (tag = rank)" if world > 1 else "1 GPU",
                           "l2": "flushed between steps (512 MB write)", "launch": tune, "tuning": tuning,
                           "numbering": args.renumber, "renumbered": renumbered},
                "step_ms_each": step_ms, "ms_per_step_median": statistics.median(step_ms), "walks_per_s": walks_s,
                "steps_per_walk": steps_per_pass / max(walks_per_pass, 1),
                "draws_per_s": draws_per_pass * args.steps * world / T_max,
                "steps_counted": "plain-equivalent walks*2^32/T" if wl["segments"] else "draws (one per step)",
                "roofline": roofline, "probe": probe, "cpu_baseline": cpu, "e2e": e2e, "plain_kernel": plain,
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
