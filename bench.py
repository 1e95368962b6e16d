"""Benchmark: direction-optimised BFS on R-MAT scale 22 (edge factor 16,
a=.57 b=.19 c=.19 d=.05, symmetrised, duplicates and self-loops removed,
seed 2) from 64 seeded random non-isolated sources, one GB300.

A step = one BFS from each of the 64 sources (the Graph500-style batch);
value = 64 * m_stored / step time in GTEPS (TEPS counts stored nonzeros as
the paper's Table 12 does), which equals the harmonic mean of the per-BFS
TEPS. The graph (0.5 GB of column indices) is larger than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the oracle (plain single-threaded C queue BFS) on
the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE, EF, SEED, NSRC, SRC_SEED = 22, 16, 2, 64, 1
METRIC = "BFS GTEPS (R-MAT s22 ef16, 64 sources, direction-optimised)"
WORKLOAD = "rmat_s22_e16_seed2_bfs64"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if s[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# Sources of the BFS kernel whose code (comments and blank lines aside) the
# DRAM traffic record in the kernel's profile summary was measured on.
BFS_KERNEL_SOURCES = ["paper_1908_01407_gb300/csrc/bfs.cu", "paper_1908_01407_gb300/csrc/bfs_common.cuh",
                      "paper_1908_01407_gb300/csrc/frontier.cuh", "paper_1908_01407_gb300/csrc/common.cuh"]
BFS_PROFILE = "profiles/k_bfs_rmat_s22.md"


def code_digest(paths, root=None):
    """sha256 of the code of `paths` (relative to root, default the
    repository) with comments and blank lines removed."""
    import hashlib
    import re
    root = ROOT if root is None else root
    h = hashlib.sha256()
    for p in paths:
        src = open(os.path.join(root, p)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for line in src.splitlines():
            line = line.strip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(profile, sources, beta=None, shape=None, alg_per_launch=None):
    """DRAM bytes per launch from a profile summary's `traffic-record` line
    for this push/pull threshold and tile shape ("pull width,blocks per SM"),
    or None when the kernel's code changed since that capture or no capture
    used this threshold and shape. A record of a sample of the sources that
    also gives the sample's mean algorithmic bytes (alg_per_launch=) is
    scaled to the caller's mean algorithmic bytes per launch."""
    try:
        text = open(os.path.join(ROOT, profile)).read()
    except OSError:
        return None
    for line in text.splitlines():
        if line.startswith("traffic-record:"):
            kv = dict(x.split("=", 1) for x in line.split(":", 1)[1].split())
            if kv.get("digest") == code_digest(sources) and (beta is None or kv.get("beta") == str(beta)) \
                    and (shape is None or kv.get("shape", "2,0") == shape):
                t = float(kv["bytes_per_launch"])
                if "alg_per_launch" in kv and alg_per_launch:
                    t *= alg_per_launch / float(kv["alg_per_launch"])
                return t
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws):
    """The slowest rank's value of x (timings are the maximum over ranks);
    x itself when there is one rank. Collective over the default group."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gteps(ws, bfs_per_rank, m, seconds):
    """GTEPS of the whole job: every replica traverses bfs_per_rank times
    the m stored edges in `seconds` (the slowest rank's time)."""
    from paper_1908_01407_gb300.metrics import teps
    return ws * bfs_per_rank * teps(m, seconds) / 1e9


def make_inputs():
    import gen
    t = gen.rmat(SCALE, EF, seed=SEED)
    srcs = gen.sources(t, NSRC, seed=SRC_SEED)
    return t, srcs


def run_reference(args):
    """The oracle, as it stands, timed on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    t, srcs = make_inputs()
    g = oracle.csr_from_tuples(t)
    m = g.m
    per_step = max(1, args.ref_sources)
    step_times = []
    k = 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            oracle.bfs(g, int(srcs[k % len(srcs)]))
            k += 1
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            step_times.append(dt)
    tot = sum(step_times)
    value = per_step * args.steps * m / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{per_step} BFS per step of the 64 sources", "m_stored": m,
                   "n": g.n},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} single-thread queue BFS per step (sources in bench order)"},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(t, srcs, budget_s):
    """Oracle BFS on the host over as many of the sources as fit the budget."""
    import oracle
    g = oracle.csr_from_tuples(t)
    done, t0 = 0, time.perf_counter()
    while done < len(srcs) and (time.perf_counter() - t0) < budget_s:
        oracle.bfs(g, int(srcs[done]))
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done * g.m / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{done} of the 64 BFS sources, single-thread queue BFS, {dt:.1f} s"}


def run_gbx(args):
    import torch
    import paper_1908_01407_gb300 as gb
    from paper_1908_01407_gb300.metrics import teps_undirected

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = f"cuda:{local}"

    t, srcs = make_inputs()
    ctx = gb.Context(local)
    stream = torch.cuda.Stream(device=dev)
    ctx.set_stream(stream)
    # matrix build (Table 4 build: tuples -> CSR, aliased CSC, live table, component sizes), timed twice:
    # from tuples already resident on the device (the paper excludes uploads), and from host tuples
    src_d = torch.from_numpy(t.src.view(np.int32)).to(dev)
    dst_d = torch.from_numpy(t.dst.view(np.int32)).to(dev)
    build_s = []
    for _ in range(2):
        torch.cuda.synchronize()
        b0 = time.perf_counter()
        A = gb.Matrix.from_tuples(ctx, t.n, src_d, dst_d, flags=gb.SYMMETRIC)
        torch.cuda.synchronize()
        build_s.append(time.perf_counter() - b0)
        A.free()
    del src_d, dst_d
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    torch.cuda.synchronize()
    build_host_s = time.perf_counter() - b0
    n, m = A.nrows, A.nvals
    desc = gb.Descriptor(beta=args.beta) if args.beta else None
    levels = torch.empty(n, dtype=torch.int32, device=dev)
    parents = torch.empty(n, dtype=torch.int32, device=dev)
    # the push/pull threshold is picked by the autotuner on 64 sources other
    # than the benchmark's (seed 99), unless --beta fixes it
    tuned_beta = None
    if not args.beta:
        import gen
        tuned_beta, _ = gb.bfs_autotune(ctx, A, gen.sources(t, 64, seed=99))
    if args.bfs_shape:
        gb.bfs_set_shape(A, *[int(x) for x in args.bfs_shape.split(",")])
    pull_width, per_sm = gb.bfs_get_shape(A)

    # untimed pass with statistics: algorithmic bytes and levels per source
    alg, depth, pushes, pulls = [], [], [], []
    for s in srcs:
        _, _, st = gb.bfs(ctx, A, int(s), levels, parents, desc=desc, stats=True)
        alg.append(st["alg_bytes"]); depth.append(st["depth"])
        pushes.append(st["push_levels"]); pulls.append(st["pull_levels"])
    alg_per_bfs = float(np.mean(alg))

    srcs_u = srcs.astype(np.uint32)

    def step():
        for s in srcs:
            gb.bfs(ctx, A, int(s), levels, parents, desc=desc, stats=False)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    total_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    # the kernel's mean duration: the timed region's CUDA events over its
    # launches (k_bfs is the only kernel there, launched back to back on the
    # stream); events around each launch would add their own cost to every
    # traversal. The per-launch event spans of one more step give the spread.
    k_ms, k_n = total_ms, args.steps * NSRC
    ctx.profile(True)
    step()
    torch.cuda.synchronize()
    span_ms, span_n = ctx.profile_get("bfs")
    ctx.profile(False)

    total_ms = max_over_ranks(total_ms, ws)
    ms_per_step = total_ms / args.steps
    value = whole_job_gteps(ws, NSRC, m, ms_per_step / 1e3)

    # end to end through the C ABI with host buffers: one gb_bfs_batch call per step writes every
    # source's levels and parents to pinned host memory (each run's copy overlaps the next run)
    lv_h = torch.empty((NSRC, n), dtype=torch.int32, pin_memory=True)
    pa_h = torch.empty((NSRC, n), dtype=torch.int32, pin_memory=True)
    # one untimed call over every row first: the first device write into a page of
    # pinned host memory costs more than later ones, and a step rewrites the same rows
    gb.bfs_batch(ctx, A, srcs_u, lv_h, pa_h, desc=desc)
    torch.cuda.synchronize()
    e_steps = max(3, args.steps)
    if ws > 1:
        dist.barrier()
    e0 = time.perf_counter()
    e2e_steps = []
    for _ in range(e_steps):
        t_s = time.perf_counter()
        gb.bfs_batch(ctx, A, srcs_u, lv_h, pa_h, desc=desc)
        e2e_steps.append(time.perf_counter() - t_s)
    e2e_s = max_over_ranks((time.perf_counter() - e0) / e_steps, ws)
    e2e_val = whole_job_gteps(ws, NSRC, m, e2e_s)
    # the plain device-to-host copy rate into the same pinned buffers (context
    # for the end-to-end figure, which the copies bound): one copy alone, and
    # levels and parents at once on two streams, as gb_bfs_batch copies them
    src_d = torch.empty_like(lv_h, device=dev)
    lv_h.copy_(src_d, non_blocking=True)
    torch.cuda.synchronize()
    c0 = time.perf_counter()
    lv_h.copy_(src_d, non_blocking=True)
    torch.cuda.synchronize()
    d2h_gbps = lv_h.numel() * 4 / (time.perf_counter() - c0) / 1e9
    s2 = [torch.cuda.Stream(device=dev) for _ in range(2)]
    c0 = time.perf_counter()
    for hb, ss in zip((lv_h, pa_h), s2):
        with torch.cuda.stream(ss):
            hb.copy_(src_d, non_blocking=True)
    torch.cuda.synchronize()
    d2h2_gbps = 2 * lv_h.numel() * 4 / (time.perf_counter() - c0) / 1e9
    del lv_h, pa_h, src_d

    hbm, peak_kind = peaks()
    avg_kernel_ms = k_ms / max(k_n, 1)          # one launch = one traversal
    alg_per_launch = alg_per_bfs
    achieved = alg_per_launch / (avg_kernel_ms / 1e3) / 1e9
    traffic = recorded_traffic(BFS_PROFILE, BFS_KERNEL_SOURCES, args.beta or tuned_beta, f"{pull_width},{per_sm}",
                               alg_per_launch)
    dram_achieved = traffic / (avg_kernel_ms / 1e3) / 1e9 if traffic else None
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "m_stored": m, "sources": NSRC, "l2": "inputs_larger_than_l2",
                   "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "beta": args.beta or tuned_beta, "beta_from": "fixed" if args.beta else "autotuner",
                   "bfs_tile": {"pull_candidates_per_lane": pull_width, "blocks_per_sm": per_sm or "all that fit",
                                "from": "fixed" if args.bfs_shape else ("autotuner" if not args.beta else "default")}},
        "gpu_launches": int(args.steps * NSRC),
        "roofline": {"bound": "hbm", "kernel": f"k_bfs<{pull_width}>", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind, "traffic": traffic,
                     "alg_bytes_per_launch": alg_per_launch, "avg_launch_ms": avg_kernel_ms,
                     # the same launches by the DRAM bytes ncu counted (null without a matching capture)
                     "dram_achieved": dram_achieved, "dram_frac": dram_achieved / hbm if dram_achieved else None},
        "e2e": {"value": e2e_val, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_copy_gbps": d2h_gbps,
                "d2h_copy_gbps_two_streams": d2h2_gbps, "step_ms": [1e3 * x for x in e2e_steps],
                "d2h_bytes_per_step": int(NSRC * 2 * 4 * n)},
        "clocks": clk,
        "build": {"ms_device_tuples": 1e3 * min(build_s), "ms_host_tuples": 1e3 * build_host_s,
                  "what": "tuples -> sorted CSR (CSC aliased), live table, FastSV component sizes"},
        "bfs": {"median_depth": float(np.median(depth)), "mean_push_levels": float(np.mean(pushes)),
                "mean_pull_levels": float(np.mean(pulls)), "ms_per_bfs": ms_per_step / NSRC,
                "alg_bytes_per_bfs": alg_per_bfs,
                "ms_per_launch_with_event_spans": span_ms / max(span_n, 1),
                "gteps_graph500": ws * NSRC * teps_undirected(m, ms_per_step / 1e3) / 1e9},
    }
    if rank == 0 and not args.no_rows:
        legs = OracleLegs() if not args.no_cpu_baseline else None
        line["rows"] = extra_rows(args, hbm)
        if legs is not None:
            legs.finish(line["rows"])
    if rank == 0 and "rows" in line:
        for k in [k for k in line["rows"] if k.startswith("_")]:
            del line["rows"][k]
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_bench(args)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(t, srcs, args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    A.free()
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def cuda_time_ms(fn, stream):
    """Device time of fn() on `stream` (CUDA events, synchronised both sides)."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def extra_rows(args, hbm):
    """GPU measurements of the other hot-path rows on their workloads."""
    import torch
    import gen
    import paper_1908_01407_gb300 as gb
    out = {}
    stream = torch.cuda.Stream()
    ctx = gb.Context(0)
    ctx.set_stream(stream)
    # --- BFS on R-MAT s14 from its max-degree vertex (the graph is L2-resident:
    # latency per BFS and per level, not bandwidth)
    t = gen.rmat(14, 16, seed=1)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    rows, _ = A.extract_tuples()
    deg = np.bincount(np.asarray(rows, dtype=np.int64), minlength=t.n)   # stored degrees
    src = int(np.flatnonzero(deg == deg.max())[0])                        # lowest id on ties
    lv = torch.empty(t.n, dtype=torch.int32, device="cuda")
    pa = torch.empty(t.n, dtype=torch.int32, device="cuda")
    _, _, st = gb.bfs(ctx, A, src, lv, pa, stats=True)
    for _ in range(10):
        gb.bfs(ctx, A, src, lv, pa, stats=False)
    reps = 200
    ms = cuda_time_ms(lambda: [gb.bfs(ctx, A, src, lv, pa, stats=False) for _ in range(reps)], stream)
    out["_bfs_s14_levels"] = lv.cpu().numpy()
    out["bfs_s14"] = {"source": src, "us_per_bfs": 1e3 * ms / reps, "depth": st["depth"],
                      "us_per_level": 1e3 * ms / reps / max(st["depth"], 1),
                      "gteps": A.nvals / (ms / reps / 1e3) / 1e9}
    A.free()
    # --- SSSP and PageRank on R-MAT s22 (weights uniform in [1, 255])
    t = gen.rmat(SCALE, EF, seed=SEED, wmax=255)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
    n, m = A.nrows, A.nvals
    srcs = gen.sources(t, 8, seed=SRC_SEED)
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    sssp_alg = []
    for s in srcs:
        sssp_alg.append(gb.sssp(ctx, A, int(s), dist, stats=True)[2]["alg_bytes"])
    iters = []
    def sssp_all():
        for s in srcs:
            _, it = gb.sssp(ctx, A, int(s), dist)
            iters.append(it)
    ctx.profile(True)
    ms = cuda_time_ms(sssp_all, stream)
    k_ms, k_n = ctx.profile_get("sssp")
    ctx.profile(False)
    k_avg = k_ms / max(k_n, 1)
    a_sssp = float(np.mean(sssp_alg))
    out["sssp_s22"] = {"sources": len(srcs), "ms_per_sssp": ms / len(srcs), "gteps": len(srcs) * m / (ms / 1e3) / 1e9,
                       "mean_iterations": float(np.mean(iters)),
                       "roofline": {"bound": "hbm", "kernel": "k_relax", "alg_bytes_per_launch": a_sssp,
                                    "avg_launch_ms": k_avg, "achieved": a_sssp / (k_avg / 1e3) / 1e9, "peak": hbm,
                                    "unit": "GB/s", "frac": a_sssp / (k_avg / 1e3) / 1e9 / hbm}}
    rank = torch.empty(n, dtype=torch.float32, device="cuda")
    # one-time cost of the degree-ordered copy (renaming + a sorted rebuild),
    # timed apart: a PageRank of no iterations builds it and runs init and normalisation
    gb.pagerank_set_order(A, 1)
    order_ms = cuda_time_ms(lambda: gb.pagerank(ctx, A, 0.85, 0, rank, residuals=False), stream)
    # the SpMV layout for this matrix: tile (nonzeros per warp tile) and vertex order
    pr_tile, pr_order, pr_staged, _ = gb.pagerank_autotune(ctx, A)
    gb.pagerank(ctx, A, 0.85, 50, rank, residuals=False)
    ms = cuda_time_ms(lambda: gb.pagerank(ctx, A, 0.85, 50, rank, residuals=False), stream)
    # a second run with the kernel spans recorded (their events add to the run's time)
    ctx.profile(True)
    cuda_time_ms(lambda: gb.pagerank(ctx, A, 0.85, 50, rank, residuals=False), stream)
    k_ms, k_n = ctx.profile_get("pagerank_spmv")
    u_ms, u_n = ctx.profile_get("pagerank_update")
    s_ms, s_n = ctx.profile_get("pagerank_span")
    ctx.profile(False)
    spmv_ms = k_ms / max(k_n, 1)
    upd_ms = u_ms / max(u_n, 1)
    span_ms = s_ms / max(s_n, 1)
    it_ms = ms / 50          # whole iterations (SpMV, the rows that cross tiles, update, reduction)
    # the cost of one more iteration: 50 against 10 iterations, so the call's
    # fixed part (tile layout, init, final normalisation) drops out
    ms10 = cuda_time_ms(lambda: gb.pagerank(ctx, A, 0.85, 10, rank, residuals=False), stream)
    it_marginal_ms = (ms - ms10) / 40
    bytes_iter = 4.0 * m + 20.0 * n
    bytes_spmv = 4.0 * m + 8.0 * n   # column indices, x once, the row sums written
    out["_pagerank_s22_rank"] = rank.cpu().numpy()
    out["pagerank_s22"] = {"iterations": 50, "tile_nnz": pr_tile, "degree_order": pr_order,
                           "staged_ranks": pr_staged,
                           "tile_from": "autotuner", "degree_copy_build_ms": order_ms,
                           "ms_total": ms, "ms_per_iteration": it_ms, "ms_total_10_iterations": ms10,
                           "ms_per_iteration_marginal": it_marginal_ms,
                           "ms_spmv_kernel": spmv_ms, "ms_update_kernel": upd_ms, "ms_span_kernel": span_ms,
                           "gteps_per_iteration": m / (it_ms / 1e3) / 1e9,
                           "iteration_alg_bytes": bytes_iter,
                           "iteration_frac": bytes_iter / (it_ms / 1e3) / 1e9 / hbm,
                           "roofline": {"bound": "hbm", "kernel": "k_pr_tiles", "alg_bytes_per_launch": bytes_spmv,
                                        "avg_launch_ms": spmv_ms,
                                        "achieved": bytes_spmv / (spmv_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                        "frac": bytes_spmv / (spmv_ms / 1e3) / 1e9 / hbm}}
    # --- adaptive PageRank (PageRankDelta): converged vertices masked out
    prd = {}
    for eps in (1e-4, 1e-5):
        gb.pagerank_delta(ctx, A, 0.85, eps, 200, rank)
        its = []
        ms = cuda_time_ms(lambda: its.append(gb.pagerank_delta(ctx, A, 0.85, eps, 200, rank)), stream)
        _, it, _, act = its[0]
        prd[f"eps_{eps:g}"] = {"ms_total": ms, "iterations": it, "row_updates": int(act.sum()),
                               "row_updates_vs_plain_50": float(act.sum()) / (50.0 * n)}
    out["pagerank_delta_s22"] = prd
    # --- multi-source BFS: the 64 benchmark sources in one bit-frontier launch
    # (one 64-bit word of source bits per vertex), then 256 distinct sources
    # of the same seeded stream in one launch (four words per vertex)
    for k_ms in (NSRC, 256):
        bsrcs = gen.sources(t, k_ms, seed=SRC_SEED)
        lv = torch.empty((k_ms, n), dtype=torch.int32, device="cuda")
        _, st_ms = gb.bfs_multi(ctx, A, bsrcs, lv)
        ms = cuda_time_ms(lambda: gb.bfs_multi(ctx, A, bsrcs, lv, stats=False), stream)
        ab = st_ms["alg_bytes"]
        out[f"bfs_multi{k_ms}_s22"] = {
            "ms_per_batch": ms, "us_per_source": 1e3 * ms / k_ms, "gteps": k_ms * m / (ms / 1e3) / 1e9,
            "levels": st_ms["depth"], "push_levels": st_ms["push_levels"], "pull_levels": st_ms["pull_levels"],
            "roofline": {"bound": "hbm", "kernel": f"k_msbfs<{(k_ms + 63) // 64}>", "alg_bytes_per_launch": ab,
                         "achieved": ab / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": ab / (ms / 1e3) / 1e9 / hbm}}
        del lv
    A.free()
    del t
    # --- triangle counting on R-MAT s20 (degree ordered, L = tril)
    t = gen.rmat(20, 16, seed=4)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
    B, _ = A.degree_order()
    L = B.tril()
    cnt = gb.tc(ctx, L)
    ms = cuda_time_ms(lambda: gb.tc(ctx, L), stream)
    out["tc_s20"] = {"triangles": cnt, "ms": ms, "nnz_L": L.nvals, "mteps": A.nvals / (ms / 1e3) / 1e6}
    for x in (A, B, L):
        x.free()
    del t
    # --- 4096 x 4096 grid, 10% of edges deleted, weights in [1, 1000]
    t = gen.grid(4096, 4096, 0.1, seed=3, wmax=1000)
    A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
    src = gen.first_nonisolated(t)
    lvg = torch.empty(t.n, dtype=torch.int32, device="cuda")
    pag = torch.empty(t.n, dtype=torch.int32, device="cuda")
    # the autotuner picks the push/pull threshold and the schedule (persistent
    # grid or single cluster) for this graph, on its own source
    beta_g, _ = gb.bfs_autotune(ctx, A, np.array([src], np.uint32))
    _, _, st = gb.bfs(ctx, A, src, lvg, pag)
    ms = cuda_time_ms(lambda: gb.bfs(ctx, A, src, lvg, pag, stats=False), stream)
    g_out = {"bfs_ms": ms, "bfs_levels": st["depth"], "bfs_us_per_level": 1e3 * ms / max(st["depth"], 1),
             "bfs_schedule": {gb.SCHED_CLUSTER: "cluster", gb.SCHED_ASYNC: "async"}.get(st["schedule"], "grid"),
             "bfs_beta": beta_g}
    d = torch.empty(t.n, dtype=torch.int32, device="cuda")
    its = []
    ms = cuda_time_ms(lambda: its.append(gb.sssp(ctx, A, src, d)[1]), stream)
    g_out.update({"sssp_ms": ms, "sssp_iterations": its[0]})
    its = []
    ms = cuda_time_ms(lambda: its.append(gb.cc(ctx, A, d)[1]), stream)
    g_out.update({"cc_ms": ms, "cc_iterations": its[0]})
    its = []
    gb.cc_fastsv(ctx, A, d)
    ms = cuda_time_ms(lambda: its.append(gb.cc_fastsv(ctx, A, d)[1]), stream)
    g_out.update({"cc_fastsv_ms": ms, "cc_fastsv_iterations": its[0]})
    # the barrier-free schedule: SSSP by distance buckets, BFS and min-label
    # components in one phase; each checked against its synchronous result
    da = gb.Descriptor(schedule=gb.SCHED_ASYNC)
    ref = torch.empty_like(d)
    gb.sssp(ctx, A, src, ref)
    _, it_a, st_a = gb.sssp(ctx, A, src, d, da, stats=True)
    ms = cuda_time_ms(lambda: gb.sssp(ctx, A, src, d, da), stream)
    ab = st_a["alg_bytes"]
    g_out["async"] = {
        "sssp_ms": ms, "sssp_buckets": it_a, "sssp_relaxations_per_vertex": st_a["vertices_reached"] / t.n,
        "sssp_matches_sync": bool(torch.equal(d, ref)),
        "sssp_roofline": {"bound": "hbm", "kernel": "k_async<SSSP>", "alg_bytes_per_launch": ab,
                          "achieved": ab / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                          "frac": ab / (ms / 1e3) / 1e9 / hbm}}
    gb.bfs(ctx, A, src, lvg, False, stats=False)
    ref.copy_(lvg)
    _, _, st_b = gb.bfs(ctx, A, src, lvg, pag, desc=da)
    ms = cuda_time_ms(lambda: gb.bfs(ctx, A, src, lvg, pag, desc=da, stats=False), stream)
    g_out["async"].update({"bfs_ms": ms, "bfs_edges_relaxed_per_stored_edge": st_b["edges_examined"] / A.nvals,
                           "bfs_matches_sync": bool(torch.equal(lvg, ref))})
    gb.cc_fastsv(ctx, A, ref)
    _, st_c = gb.cc_async(ctx, A, d, stats=True)
    ms = cuda_time_ms(lambda: gb.cc_async(ctx, A, d), stream)
    g_out["async"].update({"cc_ms": ms, "cc_relaxations_per_vertex": st_c["vertices_reached"] / t.n,
                           "cc_matches_fastsv": bool(torch.equal(d, ref))})
    da.free()
    out["grid_4096"] = g_out
    A.free()
    ctx.close()
    return out


def _timed(fn):
    t0 = time.perf_counter()
    r = fn()
    return r, time.perf_counter() - t0


class OracleLegs:
    """The oracle, as it stands (plain single-threaded C), timed on the host
    beside each GPU row on the same seeded input, and the FP32 PageRank's
    error against the FP64 oracle. The long legs run in host threads (each
    one C call at a time, the GIL released) while the GPU rows are measured:
    SSSP s22 runs Dijkstra from the first of its 8 sources; PageRank s22 runs
    all 50 FP64 iterations (also the reference of the error); TC s20 runs the
    node iterator once; the grid runs queue BFS, Dijkstra and union-find once
    each. BFS s14 runs after the GPU rows. Each leg uses one core."""

    def __init__(self):
        self.out = {}
        self.threads = [threading.Thread(target=f, daemon=True)
                        for f in (self._s22, self._tc, self._grid)]
        for t in self.threads:
            t.start()

    def _s22(self):
        import gen
        import oracle
        t = gen.rmat(SCALE, EF, seed=SEED, wmax=255)
        g = oracle.csr_from_tuples(t)
        srcs = gen.sources(t, 8, seed=SRC_SEED)
        del t
        _, dt = _timed(lambda: oracle.sssp(g, int(srcs[0])))
        self.out["sssp_s22"] = {"value": g.m / dt / 1e9, "unit": "GTEPS", "ms_per_sssp": 1e3 * dt, "cores": 1,
                                "kind": "oracle", "sample": "binary-heap Dijkstra from the first of the 8 sources"}
        (p64, _), dt = _timed(lambda: oracle.pagerank(g, 0.85, 50))
        self.out["pagerank_s22"] = {"value": 1e3 * dt / 50, "unit": "ms per iteration", "cores": 1, "kind": "oracle",
                                    "sample": "FP64 power iteration, all 50 iterations"}
        self.out["_p64"] = p64

    def _tc(self):
        import gen
        import oracle
        t = gen.rmat(20, 16, seed=4)
        g = oracle.csr_from_tuples(t)
        del t
        cnt, dt = _timed(lambda: oracle.tc(g))
        self.out["tc_s20"] = {"value": g.m / dt / 1e6, "unit": "MTEPS", "ms": 1e3 * dt, "cores": 1, "kind": "oracle",
                              "sample": "node iterator over sorted adjacency, one count"}
        self.out["_tc"] = cnt

    def _grid(self):
        import gen
        import oracle
        t = gen.grid(4096, 4096, 0.1, seed=3, wmax=1000)
        g = oracle.csr_from_tuples(t)
        src = gen.first_nonisolated(t)
        del t
        _, dt_b = _timed(lambda: oracle.bfs(g, src))
        _, dt_s = _timed(lambda: oracle.sssp(g, src))
        _, dt_c = _timed(lambda: oracle.cc(g))
        self.out["grid_4096"] = {"bfs_ms": 1e3 * dt_b, "sssp_ms": 1e3 * dt_s, "cc_ms": 1e3 * dt_c, "cores": 1,
                                 "kind": "oracle",
                                 "sample": "queue BFS, binary-heap Dijkstra and union-find, one run each"}

    def finish(self, rows):
        """Joins the legs and adds them (and the output checks) to the GPU rows."""
        import gen
        import oracle
        t = gen.rmat(14, 16, seed=1)
        g = oracle.csr_from_tuples(t)
        src = rows["bfs_s14"]["source"]
        reps = 20
        _, dt = _timed(lambda: [oracle.bfs(g, src) for _ in range(reps)])
        rows["bfs_s14"]["cpu_baseline"] = {"value": 1e6 * dt / reps, "unit": "us per BFS", "cores": 1,
                                           "kind": "oracle", "sample": f"{reps} queue BFS from the same source"}
        rows["bfs_s14"]["levels_match_oracle"] = bool(np.array_equal(rows.pop("_bfs_s14_levels"),
                                                                     oracle.bfs(g, src)))
        for t in self.threads:
            t.join()
        for k in ("sssp_s22", "pagerank_s22", "tc_s20", "grid_4096"):
            if k in self.out and k in rows:
                rows[k]["cpu_baseline"] = dict(self.out[k], sample=self.out[k]["sample"] +
                                               " (timed in a host thread while the GPU rows ran)")
        if "_p64" in self.out and "_pagerank_s22_rank" in rows:
            p64 = self.out["_p64"]
            err = np.abs(rows.pop("_pagerank_s22_rank").astype(np.float64) - p64)
            rows["pagerank_s22"]["error_vs_fp64_oracle"] = {
                "l1": float(err.sum()), "max_abs": float(err.max()),
                "max_rel": float((err / np.maximum(p64, 1e-300)).max()), "bound_l1": 1e-5}
        if "_tc" in self.out and "tc_s20" in rows:
            rows["tc_s20"]["count_matches_oracle"] = bool(self.out["_tc"] == rows["tc_s20"]["triangles"])
        return rows


def serving_bench(args):
    """Poisson stream of BFS/SSSP/PageRank (60/30/10) requests over 64
    R-MAT graphs of scales 12..20 (log-uniform, edge factor 16, weights in
    [1, 255], graph g seeded 1000 + g), served with continuous batching,
    against the same requests run one at a time on the same GPU."""
    import torch
    import gen
    import paper_1908_01407_gb300 as gb
    ctx = gb.Context(0)
    graphs = []
    for g in range(args.serve_graphs):
        scale = 12 + gen.draw(1000 + g, 0x5343414c, 0) % 9
        t = gen.rmat(int(scale), 16, seed=1000 + g, wmax=255)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
        graphs.append((A, gen.sources(t, 64, seed=1000 + g), int(scale)))
        del t
    rng = np.random.default_rng(5)
    N = args.serve_requests
    kinds = rng.choice([gb.REQ_BFS, gb.REQ_SSSP, gb.REQ_PAGERANK], size=N, p=[0.6, 0.3, 0.1])
    gids = rng.integers(0, len(graphs), N)
    srcs = [int(graphs[g][1][rng.integers(len(graphs[g][1]))]) for g in gids]
    maxn = max(A.nrows for A, _, _ in graphs)
    outb = torch.empty(64 * maxn, dtype=torch.int32, device="cuda")
    # serial baseline: one request at a time, FIFO, whole GPU
    def run_one(i):
        A = graphs[gids[i]][0]
        if kinds[i] == gb.REQ_BFS:
            gb.bfs(ctx, A, srcs[i], outb[:A.nrows], False, stats=False)
        elif kinds[i] == gb.REQ_SSSP:
            gb.sssp(ctx, A, srcs[i], outb[:A.nrows])
        else:
            gb.pagerank(ctx, A, 0.85, 50, outb[:A.nrows].view(torch.float32), residuals=False)
        ctx.synchronize()
    for i in range(min(N, 50)):
        run_one(i)
    t0 = time.perf_counter()
    lat = []
    for i in range(N):
        a = time.perf_counter()
        run_one(i)
        lat.append((time.perf_counter() - a) * 1e6)
    serial_s = time.perf_counter() - t0
    serial = {"qps": N / serial_s, "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
              "what": "service time of each request run alone, one after another"}
    service_us = np.array(lat)

    def serial_fifo(lam, nreq, seed):
        """Latency of the one-at-a-time server under the same Poisson arrivals: a
        FIFO queue whose service times are the measured ones, in request order."""
        arr = np.cumsum(np.random.default_rng(seed).exponential(1.0 / lam, nreq)) * 1e6
        done, out = 0.0, []
        for i in range(nreq):
            start = max(done, arr[i])
            done = start + service_us[i % len(service_us)]
            out.append(done - arr[i])
        return float(np.percentile(out, 50)), float(np.percentile(out, 99))
    # served: Poisson arrivals at lam = load * serial capacity
    import threading

    def run_served(load, nreq, seed):
        lam = load * serial["qps"]
        S = gb.Server(ctx, max_inflight=args.serve_slots, batch_window_us=args.serve_window_us)
        ids = [S.add_graph(A) for A, _, _ in graphs]
        arrivals = np.cumsum(np.random.default_rng(seed).exponential(1.0 / lam, nreq))
        tickets = [None] * nreq

        def fetcher():
            for i in range(nreq):
                while tickets[i] is None:
                    time.sleep(0.0002)
                r = S.wait(tickets[i], 600000)
                S.fetch_into(tickets[i], outb[:r.n])
        th = threading.Thread(target=fetcher)
        th.start()
        t0 = time.perf_counter()
        for i in range(nreq):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            tickets[i] = S.submit(int(kinds[i]), ids[gids[i]], srcs[i])
        th.join()
        st = S.stats()
        S.destroy()
        return lam, st

    lam, st = run_served(args.serve_load, N, 6)
    # latency against offered load (the first requests of the same stream), served
    # and one-at-a-time (FIFO over the measured service times, same arrivals)
    sweep = []
    for load in (0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0):
        nreq = min(N, args.serve_sweep_requests)
        lam_s, st_s = run_served(load, nreq, 7)
        s50, s99 = serial_fifo(lam_s, nreq, 7)
        sweep.append({"load": load, "offered_qps": lam_s, "qps": st_s["qps"], "p50_us": st_s["p50_us"],
                      "p99_us": st_s["p99_us"], "serial_p50_us": s50, "serial_p99_us": s99, "requests": nreq})
    target = args.serve_p99_target_ms * 1e3
    ok_served = [p for p in sweep if p["p99_us"] <= target and p["qps"] >= 0.97 * p["offered_qps"]]
    ok_serial = [p for p in sweep if p["serial_p99_us"] <= target and p["load"] < 1.0]
    at_target = {"p99_target_ms": args.serve_p99_target_ms,
                 "served_qps": max((p["qps"] for p in ok_served), default=None),
                 "serial_qps": max((p["offered_qps"] for p in ok_serial), default=None),
                 "what": "largest offered load of the sweep whose p99 stays under the target (served: "
                         "and which is kept up with), and the same for the one-at-a-time server"}
    if at_target["served_qps"] and at_target["serial_qps"]:
        at_target["speedup"] = at_target["served_qps"] / at_target["serial_qps"]
    for A, _, _ in graphs:
        A.free()
    ctx.close()
    return {"requests": N, "graphs": len(graphs), "mix": "60% BFS / 30% SSSP / 10% PageRank(50 it)",
            "offered_qps": lam, "served": {"qps": st["qps"], "p50_us": st["p50_us"], "p99_us": st["p99_us"],
                                           "batches": st["batches"], "bfs_batched": st["batched_bfs"],
                                           "slots": args.serve_slots},
            "serial": serial, "speedup_qps": st["qps"] / serial["qps"], "at_p99_target": at_target,
            "load_sweep": sweep}


def run_profile(args):
    """A short fixed run for profilers: build the workload of one kernel and
    launch it a few times (no timing, no CPU baseline). kinds: bfs (R-MAT
    s22, the benchmark sources), pr (PageRank on s22, a few iterations),
    prd (adaptive PageRank on s22, eps 1e-4), sssp (s22, weights in
    [1, 255]), msbfs (s22, 64 sources), tc (s20), fastsv (4096^2 grid),
    gridbfs (4096^2 grid, single-cluster schedule)."""
    import torch
    import gen
    import paper_1908_01407_gb300 as gb
    kind = args.profile
    ctx = gb.Context(0)
    k = args.profile_launches
    if kind == "async":
        side = args.profile_grid
        t = gen.grid(side, side, 0.1, seed=3, wmax=1000)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w, type_=gb.UINT32, flags=gb.SYMMETRIC)
        src = gen.first_nonisolated(t)
        dist = torch.empty(t.n, dtype=torch.int32, device="cuda")
        d = gb.Descriptor(schedule=gb.SCHED_ASYNC)
        for _ in range(k):
            gb.sssp(ctx, A, src, dist, d)
    elif kind == "gridbfs":
        t = gen.grid(4096, 4096, 0.1, seed=3)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
        src = gen.first_nonisolated(t)
        lv = torch.empty(t.n, dtype=torch.int32, device="cuda")
        d = gb.Descriptor(schedule=gb.SCHED_CLUSTER)
        for _ in range(k):
            gb.bfs(ctx, A, src, lv, False, desc=d, stats=False)
    elif kind == "fastsv":
        t = gen.grid(4096, 4096, 0.1, seed=3)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
        lab = torch.empty(t.n, dtype=torch.int32, device="cuda")
        for _ in range(k):
            gb.cc_fastsv(ctx, A, lab)
    elif kind == "tc":
        t = gen.rmat(20, 16, seed=4)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, flags=gb.SYMMETRIC)
        B, _ = A.degree_order()
        L = B.tril()
        for _ in range(k):
            gb.tc(ctx, L)
    else:
        t = gen.rmat(args.profile_scale, EF, seed=SEED, wmax=255 if kind == "sssp" else 0)
        srcs = gen.sources(t, NSRC, seed=SRC_SEED)
        A = gb.Matrix.from_tuples(ctx, t.n, t.src, t.dst, t.w if kind == "sssp" else None, type_=gb.UINT32,
                                  flags=gb.SYMMETRIC)
        if kind == "msbfs":
            srcs = gen.sources(t, args.ms_sources, seed=SRC_SEED)
        out = torch.empty(t.n * (len(srcs) if kind == "msbfs" else 1), dtype=torch.int32, device="cuda")
        out2 = torch.empty(t.n, dtype=torch.int32, device="cuda")
        desc = gb.Descriptor(beta=args.beta) if args.beta else None
        if args.bfs_shape:
            gb.bfs_set_shape(A, *[int(x) for x in args.bfs_shape.split(",")])
        if kind == "pr":
            gb.pagerank_set_tile(A, args.pr_tile)
            gb.pagerank_set_order(A, args.pr_order, args.pr_staged)
        alg = []
        for i in range(k):
            if kind == "bfs":
                _, _, st = gb.bfs(ctx, A, int(srcs[i]), out, out2, desc=desc, stats=True)
                alg.append(st["alg_bytes"])

            elif kind == "sssp":
                gb.sssp(ctx, A, int(srcs[i]), out)
            elif kind == "msbfs":
                gb.bfs_multi(ctx, A, srcs, out.view(len(srcs), t.n), stats=False)
            elif kind == "pr":
                gb.pagerank(ctx, A, 0.85, 2, out.view(torch.float32), residuals=False)
            elif kind == "prd":
                gb.pagerank_delta(ctx, A, 0.85, 1e-4, 200, out.view(torch.float32))
    torch.cuda.synchronize()
    ctx.close()
    if kind == "bfs":
        print(json.dumps({"alg_bytes_per_launch": alg}))

    print(f"profile run done: {kind} x{k}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbx", choices=["gbx", "reference"])
    ap.add_argument("--beta", type=int, default=0)
    ap.add_argument("--bfs-shape", default="",
                    help="BFS tile shape 'pull width,blocks per SM' (default: the autotuner's, or 2,0 with --beta)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-sources", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the SSSP/PageRank/TC/grid/multi-BFS rows")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-graphs", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-load", type=float, default=2.0, help="offered load as a multiple of serial capacity")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-window-us", type=int, default=300)
    ap.add_argument("--serve-p99-target-ms", type=float, default=25.0,
                    help="latency target of the queries/s-at-p99 figure")
    ap.add_argument("--serve-sweep-requests", type=int, default=800,
                    help="requests per point of the latency-vs-load sweep")
    ap.add_argument("--profile", choices=["bfs", "pr", "sssp", "msbfs", "tc", "prd", "fastsv", "gridbfs", "async"],
                    default=None,
                    help="short fixed run of one kernel for ncu")
    ap.add_argument("--profile-launches", type=int, default=3)
    ap.add_argument("--ms-sources", type=int, default=NSRC,
                    help="sources of the profiled multi-source BFS (up to 256 share one launch)")
    ap.add_argument("--pr-tile", type=int, default=256, help="PageRank tile of the profiled run (256, 512, 1024)")
    ap.add_argument("--pr-order", type=int, default=0,
                    help="PageRank vertex order of the profiled run (1: the degree-ordered copy)")
    ap.add_argument("--pr-staged", type=int, default=0,
                    help="ranks staged in shared memory in the profiled run (degree order; 0 = default)")
    ap.add_argument("--profile-grid", type=int, default=4096,
                    help="side of the grid of the profiled barrier-free SSSP (async)")
    ap.add_argument("--profile-scale", type=int, default=SCALE,
                    help="R-MAT scale of the profiled workload (smaller for a first pass-count check)")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gbx(args)


if __name__ == "__main__":
    main()
