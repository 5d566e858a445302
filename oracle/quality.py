"""FP64 / FP32 CPU oracle for the paper's layout quality metrics (Sec. 4,
"Quality Metrics Comparison"): neighbourhood preservation and stress.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Neighbourhood preservation, r = 2 (the paper's NP): for a vertex v,
N_G(v, 2) is the set of vertices within two hops and N_D(v, 2) the same
number of vertices nearest to v in the drawing; v scores the Jaccard index
|N_G cap N_D| / |N_G cup N_D|.  Readings:
- v itself is in neither set.
- NP is the mean of the scores: the paper prints a sum but states that NP
  lies between 0 and 1.  Vertices with an empty 2-hop ball are skipped.
- "Nearest" compares squared distances in FP32, each operation rounded on
  its own: dx = x_u - x_v, dy = y_u - y_v, dx*dx + dy*dy (no fused
  multiply-add), ties broken by the smaller vertex id.  The GPU takes the
  same decisions in the same precision.
- Both sets have b = |N_G| members, so the union has 2b - c members where c
  is the size of the intersection.
- Every vertex counts, hubs of scale-free graphs and their neighbours
  included (the paper averages over all vertices).

Stress (the paper's ST): the mean over ordered pairs i != j of
((d_ij - ||X_i - X_j||) / d_ij)^2 with d_ij the hop distance.  Readings:
- The drawing's scale is free, so it is first multiplied by the factor that
  minimises ST: with r_ij = ||X_i - X_j|| / d_ij, alpha = sum r / sum r^2
  and ST = 1 - (sum r)^2 / (N sum r^2) over the N counted pairs.
- Pairs in different components are skipped (and counted).
- With a list of source vertices, the sum runs over the pairs (s, j),
  j != s, for s in the list: all vertices give the paper's ST, a sample an
  estimate of it.
"""
from __future__ import annotations

import numpy as np

from . import pmds

def two_hop_ball(row_ptr, col, v: int) -> np.ndarray:
    """Vertices u != v with hop distance at most 2 from v (sorted ids)."""
    nb = col[row_ptr[v]:row_ptr[v + 1]].astype(np.int64)
    parts = [nb] + [col[row_ptr[w]:row_ptr[w + 1]].astype(np.int64) for w in nb]
    ball = np.unique(np.concatenate(parts)) if parts else np.empty(0, np.int64)
    return ball[ball != v]


def candidate_count(row_ptr, col, v: int) -> int:
    """deg(v) + sum of deg(w) over the adjacency entries w of v."""
    nb = col[row_ptr[v]:row_ptr[v + 1]].astype(np.int64)
    deg = np.diff(row_ptr)
    return int(nb.shape[0] + deg[nb].sum())


def sq_dist32(Y32: np.ndarray, v: int) -> np.ndarray:
    """FP32 squared distances from v, every operation rounded."""
    Y32 = np.asarray(Y32, dtype=np.float32)
    dx = (Y32[:, 0] - Y32[v, 0]).astype(np.float32)
    dy = (Y32[:, 1] - Y32[v, 1]).astype(np.float32)
    return (dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)


def nearest_in_drawing(Y32, v: int, b: int) -> np.ndarray:
    """The b vertices u != v with the smallest (squared distance, id)."""
    d2 = sq_dist32(Y32, v)
    idx = np.arange(d2.shape[0])
    keep = idx != v
    order = np.lexsort((idx[keep], d2[keep]))
    return idx[keep][order[:b]]


def neighbourhood_preservation(row_ptr, col, Y32):
    """Returns (NP, b int64[n], c int64[n]) with b = |N_G(v, 2)| and
    c = |N_G cap N_D|, over every vertex."""
    n = row_ptr.shape[0] - 1
    b = np.zeros(n, dtype=np.int64)
    c = np.zeros(n, dtype=np.int64)
    scores = []
    for v in range(n):
        ball = two_hop_ball(row_ptr, col, v)
        b[v] = ball.shape[0]
        if b[v] == 0:
            continue
        near = nearest_in_drawing(Y32, v, int(b[v]))
        c[v] = np.intersect1d(ball, near).shape[0]
        scores.append(c[v] / (2 * b[v] - c[v]))
    return (float(np.mean(scores)) if scores else 0.0), b, c


def stress(row_ptr, col, Y, sources=None):
    """Returns (ST, alpha, counted pairs, skipped pairs) over the pairs
    (s, j), j != s, for s in ``sources`` (all vertices if None)."""
    n = row_ptr.shape[0] - 1
    Y = np.asarray(Y, dtype=np.float64)
    src = np.arange(n) if sources is None else np.asarray(sources, dtype=np.int64)
    s1 = s2 = 0.0
    cnt = skipped = 0
    for s in src:
        d = pmds.bfs_distances(row_ptr, col, int(s))
        ok = d > 0
        skipped += int((d < 0).sum())
        geo = np.sqrt(((Y[ok] - Y[s]) ** 2).sum(axis=1))
        r = geo / d[ok]
        s1 += r.sum()
        s2 += (r * r).sum()
        cnt += int(ok.sum())
    if cnt == 0 or s2 == 0.0:
        return 0.0, 1.0, cnt, skipped
    return 1.0 - s1 * s1 / (cnt * s2), s1 / s2, cnt, skipped
