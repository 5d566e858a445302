"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds graph generators and the initial-layout generator only: it
contains none of the L-tsNET arithmetic (no BFS, no perplexity search, no
gradient).  Every generator is deterministic given its seed and returns an
undirected, unweighted graph in CSR form with both directions stored,
adjacency lists sorted ascending, and no self-loops or duplicate edges:

    row_ptr : int64[n + 1]
    col     : int32[row_ptr[n]]

The graph families stand in for the paper's benchmark sets (Sec. 4.1: SNAP
scale-free graphs, GION RNA networks, SuiteSparse meshes), which are not
available here.  Their shapes follow the workload recipe stated in the design
notes: a 2-D mesh (4-neighbour grid), a stochastic block model, a random
geometric graph, random recursive trees and a Barabasi-Albert graph.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Graph", "csr_from_edges", "grid2d", "sbm", "sbm_powerlaw", "rgg",
    "random_recursive_tree", "barabasi_albert", "largest_component",
    "initial_layout", "graph_batch", "config_graph", "bfs_ball",
]


@dataclass
class Graph:
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.col.shape[0] // 2)


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, name: str = "") -> Graph:
    """Undirected CSR from an edge list: drops self-loops and duplicates, stores
    both directions, sorts each adjacency list ascending."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.concatenate([u, v])
    b = np.concatenate([v, u])
    key = np.sort(a * np.int64(n) + b)
    if key.shape[0]:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    rows = key // n
    cols = (key % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(row_ptr, np.ascontiguousarray(cols), name)


def grid2d(w: int, h: int) -> Graph:
    """w x h 4-neighbour mesh; vertex (x, y) has id y*w + x."""
    ids = np.arange(w * h, dtype=np.int64).reshape(h, w)
    u = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    v = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    return csr_from_edges(w * h, u, v, name=f"grid{w}x{h}")


def _er_pairs(rng: np.random.Generator, s: int, p: float) -> tuple[np.ndarray, np.ndarray]:
    """Erdos-Renyi G(s, p) edges (i < j) on local ids, exact distribution:
    the edge count is binomial and the chosen pairs are a uniform sample
    without replacement."""
    total = s * (s - 1) // 2
    if total == 0 or p <= 0.0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    m = int(rng.binomial(total, min(p, 1.0)))
    if m == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    if m > total // 2:
        idx = rng.permutation(total)[:m].astype(np.int64)
    else:
        idx = np.zeros(0, np.int64)
        while idx.shape[0] < m:
            extra = rng.integers(0, total, size=(m - idx.shape[0]) * 2 + 16, dtype=np.int64)
            idx = np.sort(np.concatenate([idx, extra]))
            idx = idx[np.concatenate([[True], idx[1:] != idx[:-1]])]
        idx = rng.permutation(idx)[:m]
    # unrank pair index -> (i, j), i < j, row-major over the upper triangle
    # row i holds pairs with j in (i, s): cumulative count c(i) = i*s - i*(i+1)/2
    i = np.floor(((2 * s - 1) - np.sqrt((2.0 * s - 1) ** 2 - 8.0 * idx)) / 2).astype(np.int64)
    ci = i * s - i * (i + 1) // 2
    # guard floating error in the closed-form row
    over = ci > idx
    while np.any(over):
        i[over] -= 1
        ci = i * s - i * (i + 1) // 2
        over = ci > idx
    nxt = (i + 1) * s - (i + 1) * (i + 2) // 2
    under = nxt <= idx
    while np.any(under):
        i[under] += 1
        ci = i * s - i * (i + 1) // 2
        nxt = (i + 1) * s - (i + 1) * (i + 2) // 2
        under = nxt <= idx
    j = i + 1 + (idx - ci)
    return i, j


def sbm(sizes, deg_in: float, n_cross: int, seed: int, name: str = "sbm") -> Graph:
    """Stochastic block model: within block b an Erdos-Renyi graph with mean
    degree ``deg_in`` (p = deg_in/(s_b-1)); ``n_cross`` edges drawn uniformly
    among pairs in different blocks."""
    rng = np.random.default_rng(seed)
    sizes = [int(s) for s in sizes]
    n = int(sum(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    us, vs = [], []
    for b, s in enumerate(sizes):
        if s < 2:
            continue
        i, j = _er_pairs(rng, s, deg_in / (s - 1))
        us.append(i + offs[b])
        vs.append(j + offs[b])
    block = np.repeat(np.arange(len(sizes)), sizes)
    got_u, got_v = [], []
    need = int(n_cross)
    while need > 0:
        a = rng.integers(0, n, size=2 * need + 16)
        c = rng.integers(0, n, size=2 * need + 16)
        ok = block[a] != block[c]
        a, c = a[ok][:need], c[ok][:need]
        got_u.append(a)
        got_v.append(c)
        need -= a.shape[0]
    if got_u:
        us.append(np.concatenate(got_u))
        vs.append(np.concatenate(got_v))
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    return csr_from_edges(n, u, v, name=name)


def sbm_powerlaw(n: int = 100_000, blocks: int = 32, deg_in: float = 12.0,
                 deg_cross: float = 0.5, seed: int = 2) -> Graph:
    """SBM with rank-size block sizes s_b proportional to 1/(b+1) (size-density
    exponent 2), normalised to n with the remainder added to block 0; in-block
    mean degree ``deg_in``; cross-block mean degree ``deg_cross``
    (n*deg_cross/2 cross edges)."""
    w = 1.0 / np.arange(1, blocks + 1)
    sizes = np.floor(n * w / w.sum()).astype(np.int64)
    sizes[0] += n - int(sizes.sum())
    return sbm(sizes, deg_in, int(round(n * deg_cross / 2)), seed, name=f"sbm{n}")


def largest_component(g: Graph) -> Graph:
    """Induced subgraph on the largest connected component, vertices renumbered
    in their original order."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    n = g.n
    a = csr_matrix((np.ones(g.col.shape[0], np.int8), g.col, g.row_ptr), shape=(n, n))
    _, lab = connected_components(a, directed=False)
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    remap = -np.ones(n, np.int64)
    remap[keep] = np.arange(keep.shape[0])
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    sel = (remap[rows] >= 0) & (remap[g.col] >= 0)
    return csr_from_edges(keep.shape[0], remap[rows[sel]], remap[g.col[sel]], name=g.name + "-lcc")


def rgg(n: int = 1_000_000, mean_degree: float = 8.0, seed: int = 3, lcc: bool = True) -> Graph:
    """Random geometric graph: n points uniform in the unit square, an edge
    between points closer than r = sqrt(mean_degree / (pi n)); vertices keep
    their generation order; optionally restricted to the largest component."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = math.sqrt(mean_degree / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    g = csr_from_edges(n, pairs[:, 0], pairs[:, 1], name=f"rgg{n}")
    return largest_component(g) if lcc else g


def random_recursive_tree(n: int, seed: int) -> Graph:
    """Vertex i > 0 attaches to a uniformly random earlier vertex."""
    rng = np.random.default_rng(seed)
    if n < 2:
        return csr_from_edges(max(n, 1), np.zeros(0), np.zeros(0), name=f"rrt{n}")
    i = np.arange(1, n, dtype=np.int64)
    j = np.floor(rng.random(n - 1) * i).astype(np.int64)
    return csr_from_edges(n, i, j, name=f"rrt{n}")


def barabasi_albert(n: int, m_attach: int = 4, seed: int = 5) -> Graph:
    """Barabasi-Albert preferential attachment: start from a clique on
    m_attach+1 vertices; each later vertex links to m_attach distinct earlier
    vertices chosen with probability proportional to degree (sampling from the
    list of edge endpoints, repeated until distinct)."""
    rng = np.random.default_rng(seed)
    m0 = m_attach + 1
    cu, cv = np.triu_indices(m0, 1)
    ends = np.empty(2 * (cu.shape[0] + (n - m0) * m_attach), np.int64)
    ends[0:2 * cu.shape[0]:2] = cu
    ends[1:2 * cu.shape[0]:2] = cv
    fill = 2 * cu.shape[0]
    us = np.empty((n - m0) * m_attach, np.int64)
    vs = np.empty_like(us)
    e = 0
    draws = rng.random(8 * (n - m0) * m_attach + 64)
    dp = 0
    for v in range(m0, n):
        chosen = []
        while len(chosen) < m_attach:
            if dp >= draws.shape[0]:
                draws = rng.random(draws.shape[0])
                dp = 0
            t = int(ends[int(draws[dp] * fill)])
            dp += 1
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            us[e] = v
            vs[e] = t
            ends[fill] = v
            ends[fill + 1] = t
            fill += 2
            e += 1
    u = np.concatenate([cu, us[:e]])
    w = np.concatenate([cv, vs[:e]])
    return csr_from_edges(n, u, w, name=f"ba{n}")


def initial_layout(n: int, seed: int, sigma: float = 1e-4) -> np.ndarray:
    """Y0 ~ N(0, sigma^2) per coordinate, drawn in FP64 and rounded to FP32;
    shape (n, 2), row i = (x_i, y_i)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, 2)) * sigma).astype(np.float32)


def graph_batch(count: int = 512, nmin: int = 200, nmax: int = 20_000, seed: int = 4) -> list[Graph]:
    """Batch of graphs with sizes log-uniform in [nmin, nmax], round-robin over
    2-D grids, random recursive trees and SBMs with 4..16 equal blocks (in-block
    mean degree 9.5, cross-block mean degree 0.5)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = t % 3
        if kind == 0:
            w = max(1, int(round(math.sqrt(n))))
            h = max(1, int(round(n / w)))
            out.append(grid2d(w, h))
        elif kind == 1:
            out.append(random_recursive_tree(n, int(rng.integers(1 << 31))))
        else:
            b = int(rng.integers(4, 17))
            sizes = [n // b] * b
            sizes[0] += n - sum(sizes)
            out.append(sbm(sizes, 9.5, int(round(n * 0.5 / 2)), int(rng.integers(1 << 31)),
                           name=f"sbm{n}b{b}"))
    return out


def config_graph(name: str) -> Graph:
    """The named synthetic workloads: 'grid32' (32x32 mesh, n=1024),
    'sbm100k' (power-law SBM, n=1e5), 'rgg1m' (RGG, n=1e6, largest component),
    'ba4m' (Barabasi-Albert, n=4e6, 4 edges per new vertex)."""
    if name == "grid32":
        return grid2d(32, 32)
    if name == "sbm100k":
        return sbm_powerlaw()
    if name == "rgg1m":
        return rgg()
    if name == "ba4m":
        return barabasi_albert(4_000_000, 4, seed=5)
    raise KeyError(name)


def bfs_ball(g: Graph, root: int, size: int) -> tuple[Graph, np.ndarray]:
    """Induced subgraph on the first ``size`` vertices of a breadth-first
    search from ``root`` (scipy's order), relabelled in that order; returns
    (subgraph, original ids of its vertices)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order

    A = csr_matrix((np.ones(g.col.shape[0]), g.col, g.row_ptr), shape=(g.n, g.n))
    ball = breadth_first_order(A, root, directed=False, return_predecessors=False)[:size]
    new = -np.ones(g.n, np.int64)
    new[ball] = np.arange(ball.shape[0])
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    keep = (new[rows] >= 0) & (new[g.col] >= 0)
    return csr_from_edges(ball.shape[0], new[rows[keep]], new[g.col[keep]], name=f"{g.name}_ball{size}"), ball
