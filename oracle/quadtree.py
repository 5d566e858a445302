"""Oracle for the quadtree (Barnes-Hut) sums of BH-tsNET (Alg. 1) and
FIt-tsNET (Alg. 2).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

BH-tsNET approximates the repulsive KL sums (C1) with the quadtree of
BH-SNE, which the paper cites, and the entropy sum (C2) with the same kind of
tree (Eq. 7).  FIt-tsNET keeps the grid interpolation for C1 and uses the
quadtree for C2 only.  For every point i the tree is searched depth first;
a node N_j that "can be used as a summary" contributes |N_j| times the
kernel at its centre of mass.  For point i the sums are
    Zp_i = sum_j 1/(1 + d^2)            (Z = sum_i Zp_i)
    R_i  = sum_j (X_i - X_j)/(1 + d^2)^2
    E_i  = sum_j (X_i - X_j)/(eps + d^2)
with j a point or a summary node.  E_i uses Eq. 7 under the reading used
throughout this library: the kernel 1/(eps + d^2), and a sign that pushes
points apart.

The tree, with the readings the paper leaves open:
- Domain: the square [lo_x, lo_x + e] x [lo_y, lo_y + e], lo the minima
  over the points, e the larger of the two extents (1 if both are 0).  All
  of this is in FP32.
- Cells: depth 16.  A point's cell column at depth 16 is
  min(65535, floor((x - lo_x) * s)), with s = 65536 / e, in FP32 with
  every operation rounded on its own; the same for rows.  Its Morton code
  interleaves the column (even bits) and row (odd bits).  A node at depth l
  holds the points whose codes share their top 2l bits, and its cell width
  is w_l = e * 2^-l.  Nodes of one point are not split further.
- Centre of mass: exact, from fixed point.  q = rint((x - lo_x) * 2^36 / e)
  in FP64 (int64), summed over the node, then
  c = lo_x + (sum q / |N|) * (e * 2^-36) in FP64, rounded to FP32.  A node
  of one point uses the point's own coordinates.
- Summary test (BH-SNE's): w_l^2 < theta^2 d^2, d the distance from X_i to
  the node's centre, in FP32 with every operation rounded on its own.  A
  node that contains i is always opened.  A depth-16 node that is opened
  contributes its points one by one.  theta = 0 opens everything: the sums
  are exact.
"""
from __future__ import annotations

import numpy as np

LEVELS = 16
FIX_BITS = 36
EPS_DEFAULT = 1.0 / 20.0

f32 = np.float32


def _interleave(ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    code = np.zeros(ix.shape[0], dtype=np.uint64)
    for b in range(LEVELS):
        code |= ((ix.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        code |= ((iy.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return code


class Tree:
    """The quadtree of a drawing Y32 (float32 [n, 2])."""

    def __init__(self, Y32: np.ndarray):
        Y = np.asarray(Y32, dtype=f32)
        self.Y = Y
        n = Y.shape[0]
        lo = Y.min(axis=0)
        ext = max(f32(Y[:, 0].max() - lo[0]), f32(Y[:, 1].max() - lo[1]))
        if not ext > 0:
            ext = f32(1.0)
        self.lo, self.ext = lo.astype(f32), f32(ext)
        s = f32(f32(65536.0) / self.ext)
        ix = np.minimum(65535, np.floor((Y[:, 0] - self.lo[0]).astype(f32) * s).astype(np.int64))
        iy = np.minimum(65535, np.floor((Y[:, 1] - self.lo[1]).astype(f32) * s).astype(np.int64))
        self.code = _interleave(ix, iy)
        scale = 2.0 ** FIX_BITS / float(self.ext)
        self.qx = np.rint((Y[:, 0].astype(np.float64) - float(self.lo[0])) * scale).astype(np.int64)
        self.qy = np.rint((Y[:, 1].astype(np.float64) - float(self.lo[1])) * scale).astype(np.int64)
        self.order = np.lexsort((np.arange(n), self.code))  # by code, then id
        self.pos = np.empty(n, dtype=np.int64)
        self.pos[self.order] = np.arange(n)
        sc = self.code[self.order]
        # nodes[l] = list of (start, end) over sorted positions; kids[(l, a, b)]
        # = the depth-(l+1) nodes inside node (a, b) of depth l, in code order
        self.nodes = [[(0, n)]]
        self.kids = {}
        for l in range(1, LEVELS + 1):
            shift = np.uint64(2 * (LEVELS - l))
            level = []
            for (a, b) in self.nodes[l - 1]:
                if b - a <= 1:
                    continue
                pre = sc[a:b] >> shift
                cut = np.flatnonzero(pre[1:] != pre[:-1]) + 1
                edges = np.concatenate([[0], cut, [b - a]])
                ch = [(a + int(edges[t]), a + int(edges[t + 1])) for t in range(edges.shape[0] - 1)]
                self.kids[(l - 1, a, b)] = ch
                level.extend(ch)
            self.nodes.append(level)

    def centre(self, a: int, b: int) -> np.ndarray:
        if b - a == 1:
            return self.Y[self.order[a]]
        ids = self.order[a:b]
        step = float(self.ext) * 2.0 ** -FIX_BITS
        cx = float(self.lo[0]) + (float(self.qx[ids].sum()) / float(b - a)) * step
        cy = float(self.lo[1]) + (float(self.qy[ids].sum()) / float(b - a)) * step
        return np.array([cx, cy], dtype=f32)

    def children(self, l: int, a: int, b: int):
        return self.kids.get((l, a, b), [])


def _sq32(xi: np.ndarray, c: np.ndarray) -> f32:
    dx = f32(xi[0] - c[0])
    dy = f32(xi[1] - c[1])
    return f32(f32(dx * dx) + f32(dy * dy))


def sums(Y32: np.ndarray, theta: float, eps: float = EPS_DEFAULT, tree: Tree | None = None):
    """(Zp [n], R [n, 2], E [n, 2]) in FP64 by the quadtree search."""
    t = tree or Tree(Y32)
    Y = t.Y
    n = Y.shape[0]
    th2 = f32(f32(theta) * f32(theta))
    Zp = np.zeros(n)
    R = np.zeros((n, 2))
    E = np.zeros((n, 2))
    for i in range(n):
        xi = Y[i]
        xi64 = xi.astype(np.float64)
        pi = t.pos[i]
        stack = [(0, 0, n)]

        def add(c, cnt):
            d = xi64 - c.astype(np.float64)
            d2 = float(d @ d)
            q = 1.0 / (1.0 + d2)
            Zp[i] += cnt * q
            R[i] += cnt * q * q * d
            E[i] += cnt * d / (eps + d2)

        while stack:
            l, a, b = stack.pop()
            inside = a <= pi < b
            if inside and b - a == 1:
                continue
            if not inside:
                if b - a == 1:
                    add(Y[t.order[a]], 1)
                    continue
                c = t.centre(a, b)
                w = f32(t.ext * f32(2.0 ** -l))
                if f32(w * w) < f32(th2 * _sq32(xi, c)):
                    add(c, b - a)
                    continue
            if l == LEVELS:
                for p in range(a, b):
                    if p != pi:
                        add(Y[t.order[p]], 1)
                continue
            for nd in reversed(t.children(l, a, b)):
                stack.append((l + 1, nd[0], nd[1]))
    return Zp, R, E


def gradient(Y32, P_row, P_col, P_val, st, theta: float, variant: str = "bh", eps: float = EPS_DEFAULT,
             grid_parts=None):
    """BH-tsNET ("bh") or FIt-tsNET ("fit") gradient.  "bh": A exact, Z, R, E
    from the quadtree.  "fit": A, R, Z from ``grid_parts`` = (A, R, Z), the
    grid interpolation's, and E from the quadtree."""
    import oracle

    Y64 = np.asarray(Y32, dtype=np.float64)
    n = Y64.shape[0]
    Zp, R, E = sums(Y32, theta, eps)
    if variant == "bh":
        A = oracle.attractive(np.asarray(Y32, dtype=f32), P_row, P_col, P_val)
        Z = float(Zp.sum())
    else:
        A, R, Z = grid_parts
    S = float(np.sum(np.asarray(P_val, np.float64)))
    return oracle.assemble(Y64, A, R, E, Z, S, st, n), dict(A=A, R=R, E=E, Z=Z, S=S)
