"""Run L-tsNET on a seeded synthetic graph and report time and final cost.

  python -m paper_2509_19785_gb300.demo --graph rgg --n 200000 --iters 1000

Graphs: grid (sqrt(n) x sqrt(n) mesh), rgg (random geometric graph, mean
degree 8, largest component), sbm (power-law block sizes), ba
(Barabasi-Albert, 4 edges per vertex), tree (random recursive tree).
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
    args = ap.parse_args()
    import torch

    import paper_2509_19785_gb300 as lt
    import synth

    g = make_graph(args.graph, args.n, args.seed)
    params = lt.Params(perplexity=args.perplexity, stages=lt.default_stages(args.iters), plain=args.plain)
    Y0 = torch.from_numpy(synth.initial_layout(g.n, 1)).cuda()
    row_ptr = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    ws = lt.run_workspace(g.n, g.col.shape[0], params)
    times = []
    for _ in range(args.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Y, rc = lt.run(row_ptr, col, Y0, params, ws=ws)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    Yn = Y.cpu().numpy()
    print(json.dumps({"graph": args.graph, "n": g.n, "m": g.m, "iters": args.iters, "status": int(rc),
                      "seconds": [round(t, 4) for t in times], "iters_per_s": round(args.iters / min(times), 2),
                      "extent": float(Yn.max() - Yn.min())}))


if __name__ == "__main__":
    main()
