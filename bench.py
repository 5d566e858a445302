"""Benchmark of the L-tsNET hot path on GB300 (one JSON line on stdout).

A step is one whole L-tsNET run on the workload -- partial BFS, perplexity
calibration, symmetrisation, then every iteration of the schedule (gradient
+ move) -- with the graph and the initial layout already resident in HBM.
The metric is gradient iterations per second of the whole job (the C0
preprocessing amortised in), on a random geometric graph with n ~ 1e6.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ltsnet|reference]

--impl reference times the FP64 CPU oracle on this machine's host cores
instead (bounded sample; see the cpu_baseline key).  Under torchrun each rank
runs an independent replica (the single-graph path does not shard without an
exchange step); value = iterations of all ranks / max time over ranks.

Beside the headline (unless --no-batched): the 512-graph batched form
(graphs/s), the 4M-vertex Barabasi-Albert run, the quality of the final
layout (NP with r = 2, stress), the gradients and descent loops of
FIt-tsNET and BH-tsNET on the same P, and the Pivot MDS start (100 pivots).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "L-tsNET gradient iters/s at n=1M vs plain FP32 form; batched graphs/s"
WORKLOAD = "rgg1m"
PERPLEXITY = 30.0
ITERS = 1000
BATCH_ITERS = 750
BATCH_WORKERS = 16


def batch_caps(ns):
    """Per-graph grid caps of the batch (boxes per side): 1.5 times an
    envelope of the box counts the batch recipe's graphs reach at the end of
    their runs (grids, trees and SBMs of n in [200, 20000] reached at most 120
    boxes below n = 500 and 180 near n = 20000, growing with log n), rounded
    up to a multiple of 16.  Only memory depends on the cap: the grid itself
    follows each layout's extent, so a cap that never binds leaves every
    graph at the default box width."""
    import numpy as np
    ns = np.asarray(ns, dtype=np.float64)
    env = 120.0 + 60.0 * np.log(np.maximum(ns, 200.0) / 200.0) / np.log(100.0)
    return (np.ceil(1.5 * env / 16.0) * 16.0).astype(np.int32)
FUSED_PROFILE = os.path.join(ROOT, "profiles", "fused_update_rgg1m.md")
KERNEL_SOURCES = ("paper_2509_19785_gb300/csrc/iterate.cu", "paper_2509_19785_gb300/csrc/iter.cuh")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def ncu_traffic_per_launch():
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    if not os.path.exists(FUSED_PROFILE):
        return None
    text = open(FUSED_PROFILE).read()
    m = re.search(r"traffic_bytes_per_launch\s*=\s*([0-9.eE+]+)", text)
    k = re.search(r"kernel_source_hash\s*=\s*([0-9a-f]+)", text)
    if not m or not k or k.group(1) != kernel_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""
        else:
            self.out = ""

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (timings: the job ends with the
    slowest replica).  One rank: x itself."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, max_ms: float) -> float:
    """Whole-job throughput of independent replicas: every rank's units over
    the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def workload():
    import synth

    g = synth.config_graph(WORKLOAD)
    return g


def bench_ltsnet(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    import synth

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2509_19785_gb300 as lt

    lt.lib()
    g = workload()
    n = g.n
    params = lt.Params(perplexity=PERPLEXITY, stages=lt.default_stages(ITERS))
    row_ptr = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    Y0 = torch.from_numpy(synth.initial_layout(n, 1 + rank)).cuda()
    ws = lt.run_workspace(n, g.col.shape[0], params)
    stream = torch.cuda.current_stream()

    def step(p):
        Y, rc = lt.run(row_ptr, col, Y0, p, ws=ws)
        return Y

    def timed(p, steps, warmup, profile=False):
        for _ in range(warmup):
            step(p)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if profile:
            lt.profile_begin(lt.KERNEL_FUSED_UPDATE, steps * ITERS)
        l0 = lt.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            Y = step(p)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = lt.launch_count() - l0
        prof = lt.profile_end(lt.KERNEL_FUSED_UPDATE) if profile else None
        ms = max_over_ranks(ms, world)
        return ms, launches, prof, Y

    with ClockSampler(local) as clk:
        ms, launches, _, Y = timed(params, args.steps, args.warmup)
    clocks = clk.summary()

    # (after the headline timing, so the step's own launches come first in the
    # process: a profiler's launch window starts in them)
    # C0 alone (reported, part of every step)
    aff = lt.affinities(g.row_ptr, g.col, PERPLEXITY)
    nnz = int(aff["P"][1].numel())
    # Column format ltsnet_run streams: int16 offsets when, in the
    # breadth-first numbering it applies, every column is within 32767 of
    # its row (P has the same support as the graph's k-hop balls).
    order, inv, reordered = lt.bfs_order(g.row_ptr, g.col)
    col_bytes = 4
    nnz_streamed = None
    if reordered:
        invn = inv.cpu().numpy().astype(np.int64)
        rows = np.repeat(np.arange(n), np.diff(aff["P"][0].cpu().numpy()))
        cols = aff["P"][1].cpu().numpy().astype(np.int64)
        col_bytes = 2 if int(np.max(np.abs(invn[cols] - invn[rows]))) <= 32767 else 4
        # the packed layout pads every row to a multiple of 4 entries
        nnz_streamed = int(np.sum((np.diff(aff["P"][0].cpu().numpy()) + 3) // 4 * 4)) if col_bytes == 2 else None
    torch.cuda.synchronize()
    c0 = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lt.affinities(row_ptr, col, PERPLEXITY)
        e1.record(stream)
        torch.cuda.synchronize()
        c0.append(e0.elapsed_time(e1))
    del aff

    # per-launch duration of the fused kernel: one more step with CUDA events
    # around each launch (the per-launch events keep that step out of CUDA
    # graphs, so it is not part of the headline timing)
    _, _, prof, _ = timed(params, 1, 0, profile=True)
    Yn = Y.cpu().numpy()
    if not np.all(np.isfinite(Yn)):
        raise RuntimeError("non-finite layout")
    value = job_rate(world, args.steps * ITERS, ms)

    # plain FP32 form, same workload
    plain = lt.Params(perplexity=PERPLEXITY, stages=lt.default_stages(ITERS), plain=True)
    ms_plain, _, _, _ = timed(plain, max(1, args.steps // 2), 1)
    value_plain = job_rate(world, max(1, args.steps // 2) * ITERS, ms_plain)

    # the grid convolution as split-BF16 DFT matrix products on the tensor
    # cores (conv_mode 1), same workload and schedule
    gemm = lt.Params(perplexity=PERPLEXITY, stages=lt.default_stages(ITERS), conv_mode=1)
    ws_gemm = lt.run_workspace(n, g.col.shape[0], gemm)

    def step_gemm():
        return lt.run(row_ptr, col, Y0, gemm, ws=ws_gemm)[0]

    step_gemm()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(max(1, args.steps // 2)):
        Y_gemm = step_gemm()
    e1.record(stream)
    torch.cuda.synchronize()
    value_gemm = job_rate(world, max(1, args.steps // 2) * ITERS, max_over_ranks(e0.elapsed_time(e1), world))

    # grid phase per iteration (one step each with per-launch events: the
    # kernels run one after the other, the kernel spectra no longer beside
    # the spread)
    def phase_us(p, kernel, wsx):
        lt.profile_begin(kernel, ITERS)
        lt.run(row_ptr, col, Y0, p, ws=wsx)
        tot, cnt = lt.profile_end(kernel)
        return round(tot * 1e3 / max(1, cnt), 1)

    grid_phase = {"spread": phase_us(params, lt.KERNEL_SPREAD, ws),
                  "conv_fft": phase_us(params, lt.KERNEL_CONV, ws),
                  "conv_dft_gemm": phase_us(gemm, lt.KERNEL_CONV, ws_gemm),
                  "unit": "us per iteration (mean over the 1000 iterations of one step)",
                  "note": "convolution with the kernel spectra, measured with per-launch events"}
    del ws_gemm

    # end to end through the C ABI with host buffers (copies inside the region)
    Yh0 = synth.initial_layout(n, 1 + rank)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        Yh = Yh0.copy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lt.run_host(g.row_ptr, g.col, Yh, params, ws=ws)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_total = max_over_ranks(sum(e2e_ms), world)
    e2e_value = job_rate(world, args.steps * ITERS, e2e_total)

    # roofline of the fused gather + attraction + compression + update kernel
    peaks = measured_peaks()
    bytes_per_launch = 8 * nnz + 8 * (n + 1) + 48 * n  # the per-entry and per-vertex figures of the method
    # what this P format streams: entries (padded rows when packed), row
    # pointers, and per vertex the layout read, the new layout, update and
    # gains read and written
    moved_per_launch = (col_bytes + 4) * (nnz_streamed or nnz) + 8 * (n + 1) + 48 * n
    fused_ms, fused_launches = prof
    avg_s = fused_ms / 1e3 / max(1, fused_launches)
    achieved = bytes_per_launch / avg_s / 1e9
    roofline = {"kernel": "k_fused (gather + attraction + compression + update)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": ncu_traffic_per_launch(),
                "algorithmic_bytes_per_launch": bytes_per_launch, "moved_bytes_per_launch": moved_per_launch,
                "column_format": "packed rows, int16 offsets from the row" if col_bytes == 2 else "int32 (CSR)",
                "avg_launch_us": round(avg_s * 1e6, 2),
                "launches_timed": fused_launches, "peak_source": peaks["source"]}

    # quality of the final layout (Sec. 4 metrics): NP over all vertices,
    # stress over 64 sampled sources
    qual = None
    if not args.no_batched:
        qws = lt.quality_workspace(n, g.col.shape[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        npv = lt.neighbourhood_preservation(row_ptr, col, Y, ws=qws)
        torch.cuda.synchronize()
        t_np = time.perf_counter() - t0
        src = torch.from_numpy(np.random.default_rng(11).choice(n, 64, replace=False).astype(np.int32)).cuda()
        t0 = time.perf_counter()
        st, alpha, pairs, skipped = lt.stress(row_ptr, col, Y, sources=src, ws=qws)
        t_st = time.perf_counter() - t0
        qual = {"np_r2": round(npv, 5), "np_vertices": n, "np_ms": round(t_np * 1e3, 2),
                "stress": round(st, 5), "stress_sources": 64, "stress_pairs": pairs, "stress_ms": round(t_st * 1e3, 2),
                "layout": "final layout of the timed run (1000 iterations from the random start)"}
        del qws

    # the paper's three algorithms' gradients at the final layout, same P:
    # L-tsNET (grid for C1 and C2), FIt-tsNET (grid for C1, quadtree for C2),
    # BH-tsNET (quadtree for both), theta = 0.5
    variants = None
    if not args.no_batched:
        Pv = lt.affinities(row_ptr, col, PERPLEXITY)["P"]
        stv = lt.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
        gws = None
        times = {}
        for name, fn in (("ltsnet", lambda: lt.gradient(Pv, Y, stv, params)),
                         ("fit_tsnet", lambda: lt.gradient_quadtree(Pv, Y, stv, params, theta=0.5, variant="fit")),
                         ("bh_tsnet", lambda: lt.gradient_quadtree(Pv, Y, stv, params, theta=0.5, variant="bh"))):
            fn()
            ts = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            times[name] = round(statistics.median(ts) * 1e3, 3)
        # descent loops of Alg. 1 / Alg. 2 (ltsnet_optimize_quadtree), 20 steps
        # from the final layout; L-tsNET's own rate is the headline value
        loop = {}
        for vname in ("fit", "bh"):
            Yv = Y.clone()
            uv, gv = torch.zeros_like(Yv), torch.ones_like(Yv)
            lt.optimize_quadtree(Pv, Yv, uv, gv, 250, 2, params, theta=0.5, variant=vname)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lt.optimize_quadtree(Pv, Yv, uv, gv, 252, 20, params, theta=0.5, variant=vname)
            torch.cuda.synchronize()
            loop[vname + "_tsnet"] = round(20 / (time.perf_counter() - t0), 2)
            del Yv, uv, gv
        variants = {"gradient_ms": times, "optimize_iters_per_s": loop, "theta": 0.5, "n": n,
                    "note": "gradient: one call each (host-synchronous), final layout; optimize: 20 steps from it"}
        del Pv

    # Pivot MDS start (first step of Alg. 1-3) on the same graph, 100 pivots
    pm = None
    if not args.no_batched:
        k_piv = 100
        pws = lt.pivot_mds_workspace(n, k_piv)
        lt.pivot_mds(row_ptr, col, k_piv, ws=pws)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Yp, piv, eig, dist_rows = lt.pivot_mds(row_ptr, col, k_piv, ws=pws, return_dist=True)
        torch.cuda.synchronize()
        tp = max_over_ranks(time.perf_counter() - t0, world)
        finite = torch.where(dist_rows == 0xFFFF, 0, dist_rows.to(torch.int32))
        levels = int((finite.max(dim=1).values + 1).sum())
        pm = {"ms": round(tp * 1e3, 2), "pivots": k_piv, "n": n, "bfs_levels_total": levels,
              "us_per_level": round(tp * 1e6 / levels, 3), "eigvals": [float(eig[0]), float(eig[1])],
              "workspace_bytes": int(pws.numel()),
              "note": "max-min pivots: 100 sequential BFS runs of about 1000 levels each, one launch per level"}
        del pws, Yp, piv, dist_rows, finite

    # batched form: 512 independent graphs (grids, recursive trees, SBMs,
    # n log-uniform in [200, 20000]), 750 iterations each, one call
    batched = None
    if not args.no_batched:
        gs = synth.graph_batch(512)
        y0s = [synth.initial_layout(gb.n, 100 + i) for i, gb in enumerate(gs)]
        # every graph's grid arrays sized for its own cap (the arrays of the
        # whole batch live side by side); max_boxes_used says whether a cap
        # bound on any graph
        import tempfile

        caps = batch_caps([gb.n for gb in gs])
        bparams = lt.Params(perplexity=PERPLEXITY, stages=lt.default_stages(BATCH_ITERS))
        tune_cache = os.path.join(tempfile.gettempdir(), "ltsnet_autotune.json")
        fb, sb, tune_ms = lt.autotune_batched(gs, y0s, bparams, cache=tune_cache, workers=BATCH_WORKERS,
                                              max_boxes=caps)
        lt.run_batched(gs[:32], y0s[:32], bparams, workers=BATCH_WORKERS, fft_blocks=fb, spread_blocks=sb,
                       max_boxes=caps[:32])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        Yb, _, boxes = lt.run_batched(gs, y0s, bparams, workers=BATCH_WORKERS, fft_blocks=fb, spread_blocks=sb,
                                      return_boxes=True, max_boxes=caps)
        torch.cuda.synchronize()
        tb = max_over_ranks(time.perf_counter() - t0, world)
        if not bool(torch.isfinite(Yb).all()):
            raise RuntimeError("non-finite batched layout")
        del Yb
        # the same batch as stacked single-graph runs (ltsnet_run per graph on
        # the worker threads)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Yp, _ = lt.run_batched(gs, y0s, bparams, workers=BATCH_WORKERS, mode=lt.BATCH_PER_GRAPH, max_boxes=caps)
        torch.cuda.synchronize()
        tp = max_over_ranks(time.perf_counter() - t0, world)
        del Yp
        batched = {"value": round(job_rate(world, len(gs), tb * 1e3), 2), "unit": "graphs/s", "graphs": len(gs),
                   "vertices": int(sum(gb.n for gb in gs)), "iters_per_graph": BATCH_ITERS, "seconds": round(tb, 3),
                   "form": "one launch per phase over all 512 graphs (grid.y = graph), replayed from CUDA graphs; "
                           "C0 per graph on host threads",
                   "launch_shape": {"fft_blocks_per_graph": fb, "spread_blocks_per_graph": sb,
                                    "autotune_ms_per_40_iters": tune_ms},
                   "per_graph_form": {"value": round(job_rate(world, len(gs), tp * 1e3), 2), "unit": "graphs/s",
                                      "seconds": round(tp, 3), "workers": BATCH_WORKERS,
                                      "form": "ltsnet_run per graph on host worker threads, one stream each"},
                   "speedup_over_per_graph": round(tp / tb, 3),
                   "max_boxes": {"rule": "per graph: 1.5 x an envelope of the box counts the recipe's graphs "
                                         "reach, 120 + 13.0 ln(n / 200), rounded up to 16",
                                 "min": int(caps.min()), "max": int(caps.max())},
                   "max_boxes_used": int(boxes.max()),
                   "max_used_over_cap": round(float((boxes / caps).max()), 3),
                   "graphs_at_cap": int((boxes >= caps).sum())}

    # scale-free workload: Barabasi-Albert, n = 4e6, 4 edges per new vertex,
    # perplexity 50, 1000 iterations (whole run incl. C0, one step)
    ba = None
    if not args.no_batched:
        gba = synth.config_graph("ba4m")
        torch.cuda.synchronize()
        base_mem = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        rp_ba = torch.from_numpy(gba.row_ptr).cuda()
        cl_ba = torch.from_numpy(gba.col).cuda()
        y_ba = torch.from_numpy(synth.initial_layout(gba.n, 7 + rank)).cuda()
        pba = lt.Params(perplexity=50.0, stages=lt.default_stages(ITERS))
        ws_ba = lt.run_workspace(gba.n, gba.col.shape[0], pba)
        ws_bytes_ba = ws_ba.numel()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        yb, rc = lt.run(rp_ba, cl_ba, y_ba, pba, ws=ws_ba)
        torch.cuda.synchronize()
        tba = max_over_ranks(time.perf_counter() - t0, world)
        peak = torch.cuda.max_memory_allocated()
        # the fused kernel on this graph: one more run with per-launch events
        lt.profile_begin(lt.KERNEL_FUSED_UPDATE, ITERS)
        lt.run(rp_ba, cl_ba, y_ba, pba, ws=ws_ba)
        fms, fcnt = lt.profile_end(lt.KERNEL_FUSED_UPDATE)
        del ws_ba
        aff_ba = lt.affinities(rp_ba, cl_ba, 50.0)
        P_ba = aff_ba["P"]
        del aff_ba
        nnz_ba = int(P_ba[1].numel())
        ba_bytes = 8 * nnz_ba + 8 * (gba.n + 1) + 48 * gba.n
        # the format ltsnet_run streams P in on this graph (as for rgg1m above)
        _, inv_ba, reo_ba = lt.bfs_order(rp_ba, cl_ba)
        ba_fmt = "packed rows, int32 columns"
        if reo_ba:
            invb = inv_ba.cpu().numpy().astype(np.int64)
            rows_b = np.repeat(np.arange(gba.n), np.diff(P_ba[0].cpu().numpy()))
            far_b = int(np.max(np.abs(invb[P_ba[1].cpu().numpy().astype(np.int64)] - invb[rows_b])))
            if far_b <= 32767:
                ba_fmt = "packed, int16 offsets from the row"
            del rows_b
        del inv_ba
        f_s = fms / 1e3 / max(1, fcnt)
        ba = {"value": round(job_rate(world, ITERS, tba * 1e3), 2), "unit": "iters/s", "n": gba.n, "m": gba.m,
              "nnz_P": nnz_ba, "perplexity": 50, "iters": ITERS, "seconds_incl_C0": round(tba, 3),
              "workspace_bytes": int(ws_bytes_ba), "peak_device_bytes": int(peak - base_mem),
              "status": int(rc), "note": "status 1: rows whose perplexity target is unreachable (hubs) are flagged",
              "roofline": {"kernel": "k_fused (rows of more than 2048 entries summed beforehand in chunks)",
                           "column_format": ba_fmt,
                           "bound": "hbm", "achieved": round(ba_bytes / f_s / 1e9, 1), "peak": peaks["hbm_gbs"],
                           "unit": "GB/s", "frac": round(ba_bytes / f_s / 1e9 / peaks["hbm_gbs"], 4),
                           "algorithmic_bytes_per_launch": ba_bytes, "avg_launch_us": round(f_s * 1e6, 2),
                           "launches_timed": fcnt}}
        # cfg 5's differentiable cost at the final layout: forward + backward
        # of LTsNetCost with the tensor-core convolution, recomputing the grid
        # fields in backward (nothing of size nnz kept between the passes),
        # against the stored-gradient mode
        F = lt.ltsnet_cost_fn()
        stg = lt.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
        pg = lt.Params(perplexity=50.0, conv_mode=1)
        ag = {}
        for mode in (True, False):
            Yv = yb.detach().clone().requires_grad_(True)
            Pv = P_ba[2].detach().clone().requires_grad_(True)
            F.apply(Yv, Pv, P_ba[0], P_ba[1], stg, pg, mode).backward()  # warm-up (workspaces, graph state)
            Yv.grad = None
            Pv.grad = None
            torch.cuda.synchronize()
            m0 = torch.cuda.memory_allocated()
            torch.cuda.reset_peak_memory_stats()
            t0 = time.perf_counter()
            c = F.apply(Yv, Pv, P_ba[0], P_ba[1], stg, pg, mode)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            held = torch.cuda.memory_allocated() - m0  # kept for backward
            c.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            ag["recompute" if mode else "stored"] = {
                "forward_ms": round((t1 - t0) * 1e3, 2), "backward_ms": round((t2 - t1) * 1e3, 2),
                "bytes_held_between_passes": int(held),
                "peak_bytes_above_inputs": int(torch.cuda.max_memory_allocated() - m0)}
            del Yv, Pv, c
        ag["note"] = ("LTsNetCost (Eq. 1) forward by ltsnet_cost, backward dC/dY by ltsnet_gradient and dC/dP_val by "
                      "ltsnet_grad_pvals, split-BF16 DFT-GEMM convolution, final layout of the run above")
        ba["autograd"] = ag
        del yb, rp_ba, cl_ba, y_ba, P_ba

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return None
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: random geometric graph, 1e6 points in the unit square, mean degree 8, "
                               f"largest component n={n}, m={g.m}; perplexity {PERPLEXITY:g} (k=90), {ITERS} "
                               f"iterations, 3 nodes/box, min 50 boxes",
                   "n": n, "nnz_P": nnz, "iters_per_step": ITERS, "form": "optimised (fused, deterministic spread)",
                   "step": "C0 (BFS + calibration + symmetrisation) + all iterations",
                   "l2": "inputs larger than L2: P streams 6-8 bytes x nnz = 0.6-0.8 GB per iteration", "parallelism": f"replicas{world}"},
        "vertex_iters_per_s": round(value * n, 1),
        "c0_ms": round(statistics.median(c0), 3),
        "plain_fp32": {"value": round(value_plain, 2), "unit": "iters/s", "form": "unfused, atomic spread",
                       "speedup_of_optimised": round(value / value_plain, 3)},
        "dft_gemm": {"value": round(value_gemm, 2), "unit": "iters/s",
                     "form": "optimised, grid convolution as split-BF16 (3 terms, 6 products) DFT matrix "
                             "products on the tensor cores",
                     "speedup_over_plain_fp32": round(value_gemm / value_plain, 3),
                     "ratio_to_fft_form": round(value_gemm / value, 3)},
        "grid_phase_us_per_iter": grid_phase,
        "roofline": roofline,
        "e2e": {"value": round(e2e_value, 2), "unit": "iters/s",
                "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col.nbytes + 8 * n), "d2h_bytes_per_step": 8 * n},
        "batched": batched,
        "ba4m": ba,
        "pivot_mds": pm,
        "quality": qual,
        "variants": variants,
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    line["cpu_baseline"] = cpu_baseline(g)
    line["parity_vs_oracle"] = oracle_parity(g, Y.cpu().numpy())
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return line


def oracle_parity(g, Yf, size: int = 20_000):
    """Part of the oracle leg: the error of the GPU path against the FP64
    oracle on a 20,000-vertex sample of the workload -- the breadth-first
    ball of vertex 0, drawn at the timed run's final layout.  C0 (neighbour
    lists, hops, P) and, at the last stage's weights, every gradient term of
    both convolution forms, relative L2 (the assembled gradient relative to
    the sum of its terms' norms)."""
    import numpy as np
    import torch

    import oracle
    import paper_2509_19785_gb300 as lt
    import synth

    sub, ids = synth.bfs_ball(g, 0, size)
    Y32 = np.ascontiguousarray(Yf[ids], dtype=np.float32)
    ref = oracle.preprocess(sub.row_ptr, sub.col, PERPLEXITY)
    aff = lt.affinities(sub.row_ptr, sub.col, PERPLEXITY)
    torch.cuda.synchronize()
    pv32 = aff["P"][2].cpu().numpy()
    c0 = {"nbr_equal": bool(np.array_equal(aff["nbr"].cpu().numpy(), ref.nbr)),
          "hop_equal": bool(np.array_equal(aff["hop"].cpu().numpy().astype(np.int32), ref.hop)),
          "P_pattern_equal": bool(np.array_equal(aff["P"][0].cpu().numpy(), ref.P_row)
                                  and np.array_equal(aff["P"][1].cpu().numpy(), ref.P_col)),
          "P_val_equal_fp32_of_fp64": bool(np.array_equal(pv32, ref.P_val64.astype(np.float32)))}
    pv = pv32.astype(np.float64)
    st = lt.default_stages(ITERS)[-1]
    ost = oracle.Stage(st.iters, st.lambda_kl, st.lambda_c, st.lambda_r, st.exaggeration, st.momentum)
    gref, pr = oracle.interp_gradient(Y32, ref.P_row, ref.P_col, pv, ost, oracle.GridParams())
    nn = sub.n
    scale = (np.linalg.norm(4 * ost.lambda_kl * ost.exaggeration * pr["A"])
             + np.linalg.norm(4 * ost.lambda_kl * pr["S"] / pr["Z"] * pr["R"])
             + np.linalg.norm(ost.lambda_c / nn * Y32.astype(np.float64))
             + np.linalg.norm(ost.lambda_r / nn ** 2 * pr["E"]))

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))

    forms = {}
    for name, conv in (("fft", 0), ("dft_gemm", 1)):
        grad, parts, terms = lt.gradient(aff["P"], torch.from_numpy(Y32).cuda(), st,
                                         lt.Params(perplexity=PERPLEXITY, conv_mode=conv), parts=True)
        grad, parts, terms = grad.cpu().numpy(), parts.cpu().numpy(), terms.cpu().numpy()
        forms[name] = {"A": rel(parts[:, 0:2], pr["A"]), "R": rel(parts[:, 2:4], pr["R"]),
                       "E": rel(parts[:, 4:6], pr["E"]), "Z": float(abs(terms[0] - pr["Z"]) / pr["Z"]),
                       "grad_vs_term_norms": float(np.linalg.norm(grad - gref) / scale)}
    return {"sample": f"breadth-first ball of {sub.n} vertices around vertex 0, final layout of the timed run "
                      f"(extent {float(Y32.max() - Y32.min()):.1f}, grid {pr['grid'].I} boxes per side)",
            "c0": c0, "gradient_rel_l2": forms, "tolerance": 1e-5}


def oracle_affinities(g):
    import oracle

    return oracle.preprocess(g.row_ptr, g.col, PERPLEXITY)


def oracle_iteration_time(g, aff, iters: int, lr: float):
    """Seconds per oracle iteration (interpolated gradient + update) on the
    full workload, starting from a spread layout (the loop's typical grid)."""
    import numpy as np

    import oracle

    st = oracle.default_stages(ITERS)[-1]
    Y = (np.random.default_rng(0).standard_normal((g.n, 2)) * 15).astype(np.float64)
    upd = np.zeros_like(Y)
    gains = np.ones_like(Y)
    t0 = time.perf_counter()
    for _ in range(iters):
        Y32 = Y.astype(np.float32)
        gr, _ = oracle.interp_gradient(Y32, aff.P_row, aff.P_col, aff.P_val64, st, oracle.GridParams())
        Y, upd, gains = oracle.update(Y32.astype(np.float64), upd, gains, gr, st.momentum, lr)
    return (time.perf_counter() - t0) / max(1, iters)


def cpu_baseline(g, n_sample: int = 100_000, iters: int = 3):
    """The oracle, as it stands, on a 100k-vertex instance of the same recipe
    (C0 + a few iterations), scaled linearly in n (every step is O(n)): on
    one thread and on all host cores (the oracle's row-parallel loops; its
    spread and numpy's FFT stay on one thread)."""
    import oracle
    import synth

    gs = synth.rgg(n_sample)
    cores = os.cpu_count() or 1
    out = {}
    for threads in (1, cores):
        used = oracle.set_threads(threads)
        t0 = time.perf_counter()
        aff = oracle_affinities(gs)
        c0_s = time.perf_counter() - t0
        per_iter = oracle_iteration_time(gs, aff, iters, oracle.auto_learning_rate(gs.n))
        scale = g.n / gs.n
        run_s = scale * (c0_s + ITERS * per_iter)
        out[threads] = (ITERS / run_s, used, c0_s, per_iter, scale)
    v1, _, c01, it1, scale = out[1]
    vn, used, c0n, itn, _ = out[cores]
    return {"value": round(vn, 5), "unit": "iters/s", "cores": used, "kind": "oracle",
            "sample": f"oracle on a {gs.n}-vertex RGG of the same recipe: C0 {c0n:.1f} s + {iters} iterations "
                      f"(interpolated gradient + update) {itn:.3f} s each on {used} threads, one {ITERS}-iteration "
                      f"run scaled by n ({scale:.2f}x)",
            "single_thread": {"value": round(v1, 5), "cores": 1, "c0_s": round(c01, 2), "iter_s": round(it1, 3)},
            "nproc": cores}


def bench_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import oracle
    import synth

    oracle.build()
    g = workload()
    t0 = time.perf_counter()
    aff = oracle_affinities(g)
    c0_s = time.perf_counter() - t0
    lr = oracle.auto_learning_rate(g.n)
    if args.warmup > 0:
        oracle_iteration_time(g, aff, args.warmup, lr)
    per_iter = oracle_iteration_time(g, aff, max(1, args.steps), lr)
    run_s = c0_s + ITERS * per_iter
    value = ITERS / run_s
    cb = {"value": round(value, 5), "unit": "iters/s", "cores": 1, "kind": "oracle",
          "sample": f"oracle C0 on the full graph ({c0_s:.1f} s, once) + {args.steps} timed oracle iterations "
                    f"({per_iter:.2f} s each, after {args.warmup} warm-up iterations), extrapolated to one "
                    f"{ITERS}-iteration run; single thread"}
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(run_s * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: random geometric graph n={g.n}, perplexity {PERPLEXITY:g}, "
                                   f"{ITERS} iterations", "n": g.n},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ltsnet", choices=["ltsnet", "reference"])
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 512-graph batched and the 4M-vertex Barabasi-Albert measurements")
    args = ap.parse_args()
    line = bench_reference(args) if args.impl == "reference" else bench_ltsnet(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
