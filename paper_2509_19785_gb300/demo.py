"""Run L-tsNET (or BH-tsNET / FIt-tsNET) on a seeded synthetic graph and
report the time, the layout's extent and, with --quality, its NP and stress.

  python -m paper_2509_19785_gb300.demo --graph rgg --n 200000 --iters 1000
  python -m paper_2509_19785_gb300.demo --graph rgg --n 200000 --init pmds --quality
  python -m paper_2509_19785_gb300.demo --graph rgg --n 300000 --variant bh --iters 20
  python -m paper_2509_19785_gb300.demo --graph rgg --n 1000000 --iters 30 --init uniform --extent 45 --conv gemm

Graphs: grid (sqrt(n) x sqrt(n) mesh), rgg (random geometric graph, mean
degree 8, largest component), sbm (power-law block sizes), ba
(Barabasi-Albert, 4 edges per vertex), tree (random recursive tree), batch
(--n graphs of 200..20000 vertices, grids / recursive trees / SBMs, run by
ltsnet_run_batched):

  python -m paper_2509_19785_gb300.demo --graph batch --n 512 --iters 750 --max-boxes 128
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def make_graph(kind: str, n: int, seed: int):
    import synth

    if kind == "grid":
        w = max(2, int(round(math.sqrt(n))))
        return synth.grid2d(w, max(2, n // w))
    if kind == "rgg":
        return synth.rgg(n, 8.0, seed)
    if kind == "sbm":
        return synth.sbm_powerlaw(n, 32, 12.0, 0.5, seed)
    if kind == "ba":
        return synth.barabasi_albert(n, 4, seed)
    if kind == "tree":
        return synth.random_recursive_tree(n, seed)
    raise SystemExit(f"unknown graph {kind}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graph", default="rgg")
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--perplexity", type=float, default=30.0)
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--plain", action="store_true")
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--variant", choices=["ltsnet", "fit", "bh"], default="ltsnet",
                    help="ltsnet: ltsnet_run (Alg. 3); fit / bh: C0, then ltsnet_optimize_quadtree (Alg. 2 / 1)")
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--init", choices=["random", "pmds", "uniform"], default="random",
                    help="random N(0, 1e-4^2) start, Pivot MDS with 100 pivots (the paper's start), or points "
                         "uniform in a square of side --extent (the grid sizes of a late iteration from the start)")
    ap.add_argument("--extent", type=float, default=45.0)
    ap.add_argument("--late-stage", action="store_true",
                    help="every iteration with the second stage's multipliers (lambda_c 0.01, lambda_r 0.6, "
                         "momentum 0.8): a layout that keeps its extent, for profiling late iterations")
    ap.add_argument("--conv", choices=["fft", "gemm"], default="fft",
                    help="grid convolution: FP32 FFT or split-BF16 DFT matrix products on the tensor cores")
    ap.add_argument("--quality", action="store_true", help="NP (r = 2) and stress over 64 sources of the result")
    ap.add_argument("--max-boxes", type=int, default=None, help="cap on the boxes per side of the grid")
    ap.add_argument("--batch-form", choices=["one", "per-graph"], default="one",
                    help="batch: one launch per phase over all graphs, or ltsnet_run per graph on worker threads")
    ap.add_argument("--fft-blocks", type=int, default=0, help="batch: FFT blocks per graph (0: the library's default)")
    ap.add_argument("--spread-blocks", type=int, default=0,
                    help="batch: spread blocks per graph (0: the library's default)")
    ap.add_argument("--workers", type=int, default=16, help="batch: host threads for C0 (and the per-graph form)")
    args = ap.parse_args()
    if args.graph == "batch":
        return run_batch(args)
    import torch

    import paper_2509_19785_gb300 as lt
    import synth

    g = make_graph(args.graph, args.n, args.seed)
    stages = [lt.Stage(args.iters, 1.0, 0.01, 0.6, 1.0, 0.8)] if args.late_stage else lt.default_stages(args.iters)
    params = lt.Params(perplexity=args.perplexity, stages=stages, plain=args.plain,
                       conv_mode=1 if args.conv == "gemm" else 0)
    if args.max_boxes:
        params.max_boxes = args.max_boxes
    row_ptr = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    if args.init == "pmds":
        Y0, _, _ = lt.pivot_mds(row_ptr, col, min(100, g.n))
    elif args.init == "uniform":
        import numpy as np

        Y0 = torch.from_numpy((np.random.default_rng(1).random((g.n, 2)) * args.extent).astype(np.float32)).cuda()
    else:
        Y0 = torch.from_numpy(synth.initial_layout(g.n, 1)).cuda()
    times = []
    rc = 0
    if args.variant == "ltsnet":
        ws = lt.run_workspace(g.n, g.col.shape[0], params)
        for _ in range(args.repeat):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Y, rc = lt.run(row_ptr, col, Y0, params, ws=ws)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
    else:
        P = lt.affinities(row_ptr, col, args.perplexity)["P"]
        for _ in range(args.repeat):
            Y = Y0.clone()
            upd, gains = torch.zeros_like(Y), torch.ones_like(Y)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lt.optimize_quadtree(P, Y, upd, gains, 0, args.iters, params, theta=args.theta, variant=args.variant)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
    Yn = Y.cpu().numpy()
    out = {"graph": args.graph, "n": g.n, "m": g.m, "variant": args.variant, "init": args.init, "conv": args.conv,
           "iters": args.iters, "status": int(rc), "seconds": [round(t, 4) for t in times],
           "iters_per_s": round(args.iters / min(times), 2), "extent": float(Yn.max() - Yn.min())}
    if args.quality:
        import numpy as np

        out["np_r2"] = lt.neighbourhood_preservation(row_ptr, col, Y)
        src = np.random.default_rng(11).choice(g.n, min(64, g.n), replace=False).astype(np.int32)
        out["stress"] = lt.stress(row_ptr, col, Y, sources=src)[0]
    print(json.dumps(out))


def run_batch(args):
    import numpy as np
    import torch

    import paper_2509_19785_gb300 as lt
    import synth

    gs = synth.graph_batch(args.n)
    y0s = [synth.initial_layout(g.n, 100 + i) for i, g in enumerate(gs)]
    params = lt.Params(perplexity=args.perplexity, stages=lt.default_stages(args.iters))
    if args.max_boxes:
        params.max_boxes = args.max_boxes
    mode = lt.BATCH_ONE_LAUNCH if args.batch_form == "one" else lt.BATCH_PER_GRAPH
    times = []
    boxes = None
    c0 = lt.launch_count()
    for _ in range(args.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = lt.run_batched(gs, y0s, params, workers=args.workers, mode=mode, fft_blocks=args.fft_blocks,
                             spread_blocks=args.spread_blocks, return_boxes=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        Yb, _, boxes = out
    boxes = np.asarray(boxes)
    print(json.dumps({"graph": "batch", "graphs": len(gs), "vertices": int(sum(g.n for g in gs)),
                      "form": args.batch_form, "iters": args.iters,
                      "seconds": [round(t, 4) for t in times], "graphs_per_s": round(len(gs) / min(times), 2),
                      "max_boxes_used": int(boxes.max()), "graphs_at_cap": int((boxes >= params.max_boxes).sum()),
                      "launches": lt.launch_count() - c0, "finite": bool(torch.isfinite(Yb).all())}))


if __name__ == "__main__":
    main()
