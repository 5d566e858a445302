"""FP64 CPU oracle for the Pivot MDS initial layout.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by ``tests/``
and by ``bench.py``'s CPU-baseline leg, never by the GPU library.

Every variant in the paper (BH-tsNET, FIt-tsNET and L-tsNET; Alg. 1-3, first
step) starts from a Pivot MDS layout of the graph.  Sec. 2 defines tsNET* as
tsNET with this initialisation, and Sec. 4 uses it for all experiments.  The
paper cites Brandes and Pich (GD 2006, "Eigensolver methods for progressive
multidimensional scaling of large data") for the method and gives none of its
parameters.  The method as written here:

1. Pivots by max-min: the first pivot is given.  Each further pivot is the
   vertex whose BFS distance to its nearest chosen pivot is largest.
2. D: the n x k matrix of BFS hop distances from the k pivots.
3. C = -1/2 J_n (D o D) J_k: the squared distances, double-centred over the
   vertices and over the pivots (J_m = I - 11^T/m).
4. v_1, v_2: the unit eigenvectors of C^T C (k x k) for its two largest
   eigenvalues sigma_1^2 >= sigma_2^2.
5. The coordinates are x_d = C v_d / sqrt(sigma_d).

Readings, because the paper leaves these open:
- Ties in the max-min choice go to the smallest vertex index.  A vertex that
  no chosen pivot reaches counts as infinitely far, so every component gets a
  pivot once there are enough pivots.
- A pair in different components gets distance (largest finite pivot
  distance + 1).
- The scale is 1/sqrt(sigma_d).  With it, Pivot MDS with every vertex as a
  pivot is classical (Torgerson) MDS: C = B, sigma_d = lambda_d(B), and
  C v_d / sqrt(sigma_d) = sqrt(lambda_d) v_d.  Unscaled C v_d would stretch
  axis 1 against axis 2 by sigma_1 / sigma_2.
- An axis whose eigenvalue is at most 1e-10 of the first is set to zero
  (a path graph is one-dimensional).
- Sign: each v_d is flipped so that its first entry (smallest index) whose
  magnitude is within a relative 1e-9 of the largest is positive.  The slack
  keeps the choice stable under rounding where entries tie in magnitude (a
  symmetric graph, or k = 2, where v = (1, -1)/sqrt(2)).
- Final scale: both axes are multiplied by one factor so that the layout's
  RMS distance from its centroid is sqrt(2) * init_std, i.e. the same spread as
  the N(0, init_std^2) random start (init_std = 1e-4).  init_std = 0 keeps the
  MDS scale.  The factor does not depend on a rotation of the axes, so the
  scaled layout is unique even when sigma_1 = sigma_2.

numpy's symmetric eigensolver (eigh) is the one library step.
"""
from __future__ import annotations

import numpy as np

UNREACHED = -1
AXIS_EPS = 1e-10
SIGN_SLACK = 1e-9


def bfs_distances(row_ptr: np.ndarray, col: np.ndarray, src: int) -> np.ndarray:
    """Hop distances from ``src`` by level-synchronous BFS; -1 where
    unreachable.  int64[n]."""
    n = row_ptr.shape[0] - 1
    d = np.full(n, UNREACHED, dtype=np.int64)
    d[src] = 0
    frontier = np.array([src], dtype=np.int64)
    level = 0
    while frontier.size:
        starts, ends = row_ptr[frontier], row_ptr[frontier + 1]
        lens = ends - starts
        if lens.sum() == 0:
            break
        # every edge leaving the frontier
        idx = np.repeat(starts - np.cumsum(lens) + lens, lens) + np.arange(lens.sum())
        nb = col[idx].astype(np.int64)
        nb = np.unique(nb[d[nb] == UNREACHED])
        level += 1
        d[nb] = level
        frontier = nb
    return d


def maxmin_pivots(row_ptr: np.ndarray, col: np.ndarray, k: int, first: int = 0):
    """Step 1 and 2: the k max-min pivots and their distance rows.

    Returns (pivots int64[k], D int64[k, n] with -1 for unreachable)."""
    n = row_ptr.shape[0] - 1
    if not 1 <= k <= n:
        raise ValueError("need 1 <= k <= n")
    inf = np.iinfo(np.int64).max
    nearest = np.full(n, inf, dtype=np.int64)
    piv = np.empty(k, dtype=np.int64)
    D = np.empty((k, n), dtype=np.int64)
    p = first
    for t in range(k):
        piv[t] = p
        D[t] = bfs_distances(row_ptr, col, p)
        dt = np.where(D[t] == UNREACHED, inf, D[t])
        nearest = np.minimum(nearest, dt)
        p = int(np.argmax(nearest))  # first index of the maximum
    return piv, D


def squared_distances(D: np.ndarray) -> np.ndarray:
    """D o D as FP64 n x k, with unreachable pairs at (largest finite + 1)."""
    fill = int(D.max()) + 1
    Df = np.where(D == UNREACHED, fill, D).astype(np.float64)
    return (Df * Df).T


def pmds_coords(A: np.ndarray, init_std: float = 1e-4):
    """Steps 3-5 and the final scale from the n x k squared distances A.

    Returns (Y float64[n, 2], eigenvalues sigma^2 of the two axes)."""
    n, k = A.shape
    Jn_A = A - A.mean(axis=0, keepdims=True)
    C = -0.5 * (Jn_A - Jn_A.mean(axis=1, keepdims=True))
    lam, V = np.linalg.eigh(C.T @ C)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    Y = np.zeros((n, 2))
    for d in range(2):
        if d >= k or lam[d] <= AXIS_EPS * lam[0]:
            continue
        v = V[:, d]
        a = np.abs(v)
        j = int(np.flatnonzero(a >= (1.0 - SIGN_SLACK) * a.max())[0])
        if v[j] < 0:
            v = -v
        Y[:, d] = C @ v / np.sqrt(np.sqrt(lam[d]))
    if init_std > 0:
        rms = np.sqrt((Y * Y).sum() / (2 * n))
        if rms > 0:
            Y *= init_std / rms
    return Y, lam[:2].copy()


def pivot_mds(row_ptr: np.ndarray, col: np.ndarray, k: int, first: int = 0, init_std: float = 1e-4):
    """The whole initial layout: (Y float64[n, 2], pivots, D, eigenvalues)."""
    piv, D = maxmin_pivots(row_ptr, col, k, first)
    Y, lam = pmds_coords(squared_distances(D), init_std)
    return Y, piv, D, lam
