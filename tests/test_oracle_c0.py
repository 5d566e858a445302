"""Pins of the oracle's preprocessing (C0 of Alg. 3) to independent facts:
scipy's breadth-first order, Floyd-Warshall distances, lattice closed forms,
an independent root finder for the perplexity equation and a dense-matrix
construction of Eq. 2."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import breadth_first_order

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    return synth.csr_from_edges(n, iu[keep], ju[keep])


def floyd_warshall(g):
    n = g.n
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    for i in range(n):
        D[i, g.col[g.row_ptr[i]:g.row_ptr[i + 1]]] = 1
    for m in range(n):
        D = np.minimum(D, D[:, m:m + 1] + D[m:m + 1, :])
    return D


@pytest.mark.parametrize("seed", range(12))
def test_bfs_against_floyd_warshall(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(5, 64))
    g = random_graph(n, float(rng.uniform(0.03, 0.3)), seed)
    D = floyd_warshall(g)
    k = int(rng.integers(1, n + 5))
    nbr, hop, cnt = oracle.partial_bfs(g.row_ptr, g.col, k)
    for s in range(n):
        reach = np.isfinite(D[s])
        assert cnt[s] == min(k, int(reach.sum()) - 1)
        row = nbr[s, :cnt[s]]
        assert len(set(row.tolist())) == cnt[s] and s not in row
        assert np.array_equal(hop[s, :cnt[s]], D[s, row].astype(np.int32))
        assert np.all(np.diff(hop[s, :cnt[s]]) >= 0)
        assert np.all(nbr[s, cnt[s]:] == -1)
        if cnt[s]:
            far = hop[s, cnt[s] - 1]
            closer = set(np.flatnonzero(D[s] < far).tolist()) - {s}
            assert closer <= set(row.tolist())  # distance-prefix closed


@pytest.mark.parametrize("gname", ["grid", "random", "tree", "ba"])
def test_bfs_order_is_scipy_breadth_first_order(gname):
    """The partial BFS is the prefix of a full FIFO breadth-first order that
    visits adjacency in CSR order (scipy.sparse.csgraph.breadth_first_order)."""
    g = {"grid": synth.grid2d(9, 7), "random": random_graph(80, 0.06, 3),
         "tree": synth.random_recursive_tree(150, 2), "ba": synth.barabasi_albert(200, 3, seed=1)}[gname]
    A = csr_matrix((np.ones(g.col.shape[0]), g.col, g.row_ptr), shape=(g.n, g.n))
    k = 25
    nbr, hop, cnt = oracle.partial_bfs(g.row_ptr, g.col, k)
    for s in range(g.n):
        order = breadth_first_order(A, s, directed=True, return_predecessors=False)
        want = order[1:k + 1]
        assert cnt[s] == want.shape[0]
        assert np.array_equal(nbr[s, :cnt[s]], want)


def test_bfs_lattice_closed_form():
    """Interior vertex of the 32x32 grid: the hop-r shell of the 4-neighbour
    lattice has 4r vertices, so with k = 90 the row holds all 84 vertices with
    r <= 6 and 6 of the 28 at r = 7 (tests/golden/grid32_interior_shells.txt)."""
    gold = dict(l.split("=") for l in open(os.path.join(GOLDEN, "grid32_interior_shells.txt")).read().split()
                if "=" in l)
    g = synth.grid2d(32, 32)
    k = int(gold["k"])
    nbr, hop, cnt = oracle.partial_bfs(g.row_ptr, g.col, k)
    s = 16 * 32 + 16
    counts = np.bincount(hop[s, :cnt[s]])[1:]
    assert counts.tolist() == [int(x) for x in gold["shell_counts"].split(",")]


def entropy_bits(p):
    p = np.asarray(p, np.longdouble)
    p = p[p > 0]
    return float(-np.sum(p * np.log2(p)))


def test_beta_against_independent_root_finder():
    """Grid-interior shell profile {4, 8, 12, 16, 20, 24, 6} at u = 30: the
    oracle's beta satisfies 2^(H in bits) = u to the stated tolerance, and
    agrees with a bracketing root (brentq) of the same equation written in
    base 2 in extended precision."""
    counts = [4, 8, 12, 16, 20, 24, 6]
    hop = np.concatenate([np.full(c, r + 1, np.int32) for r, c in enumerate(counts)])[None, :]
    u = 30.0
    beta, pcond, conv = oracle.calibrate(hop, np.array([hop.shape[1]], np.int32), u)

    def f(b):
        d2 = hop[0].astype(np.longdouble) ** 2
        w = np.exp(-np.longdouble(b) * (d2 - d2.min()))
        return entropy_bits(w / w.sum()) - math.log2(u)

    root = brentq(f, 1e-6, 50.0, xtol=1e-15)
    assert conv[0] == 1
    assert abs(entropy_bits(pcond[0]) * math.log(2) - math.log(u)) < 1e-5
    h = 1e-7
    slope = abs(f(root + h) - f(root - h)) / (2 * h) * math.log(2)
    assert abs(beta[0] - root) <= 1e-5 / slope * 1.01


def test_beta_above_one_against_root_finder():
    """Three vertices one hop away and a hundred two hops away at u = 5: at
    beta = 1 the mass sits mostly on the far shell (entropy about 3.3 > ln 5),
    so the search must raise beta before it brackets the root; the result
    agrees with brentq on the same equation."""
    hop = np.concatenate([np.full(3, 1, np.int32), np.full(100, 2, np.int32)])[None, :]
    u = 5.0
    beta, pcond, conv = oracle.calibrate(hop, np.array([hop.shape[1]], np.int32), u)

    def f(b):
        d2 = hop[0].astype(np.longdouble) ** 2
        w = np.exp(-np.longdouble(b) * (d2 - d2.min()))
        return entropy_bits(w / w.sum()) * math.log(2) - math.log(u)

    assert f(1.0) > 0
    root = brentq(f, 1e-6, 50.0, xtol=1e-15)
    assert root > 1.0 and conv[0] == 1
    h = 1e-7
    slope = abs(f(root + h) - f(root - h)) / (2 * h)
    assert abs(beta[0] - root) <= 1e-5 / slope * 1.01


@pytest.mark.parametrize("u", [5.0, 30.0, 40.0, 50.0])
def test_calibrated_rows_sum_to_one_with_target_entropy(u):
    g = synth.sbm([300, 200, 150], 12.0, 100, seed=4)
    k = oracle.k_from_perplexity(u)
    nbr, hop, cnt = oracle.partial_bfs(g.row_ptr, g.col, k)
    beta, p, conv = oracle.calibrate(hop, cnt, u)
    for i in range(g.n):
        c = cnt[i]
        assert abs(p[i, :c].sum() - 1.0) < 1e-12
        assert np.all(p[i, c:] == 0)
        if conv[i]:
            assert abs(entropy_bits(p[i, :c]) * math.log(2) - math.log(u)) < 1e-5
        # p is non-increasing in hop distance (beta > 0)
        assert np.all(np.diff(p[i, :c]) <= 1e-15)


def test_calibrate_unreachable_targets():
    """Sec. 4.1's "perplexity too low": a hub whose nearest shell alone holds
    more than u vertices cannot reach ln u (p becomes uniform on that shell);
    a vertex with fewer than u reachable vertices cannot either (p uniform)."""
    star = synth.csr_from_edges(61, np.zeros(60, np.int64), np.arange(1, 61))
    u = 20.0
    k = oracle.k_from_perplexity(u)
    nbr, hop, cnt = oracle.partial_bfs(star.row_ptr, star.col, k)
    beta, p, conv = oracle.calibrate(hop, cnt, u)
    # hub: 60 leaves at distance 1, k = 60 entries, uniform 1/60 > ... H = ln 60 > ln 20: beta -> inf, still uniform
    assert conv[0] == 0 and np.allclose(p[0, :cnt[0]], 1.0 / cnt[0])
    small = synth.grid2d(2, 3)
    nbr, hop, cnt = oracle.partial_bfs(small.row_ptr, small.col, k)
    beta, p, conv = oracle.calibrate(hop, cnt, u)
    assert np.all(conv == 0) and np.all(cnt == 5)
    assert np.allclose(p[:, :5], 0.2, atol=1e-12)


def test_symmetrize_against_dense_matrix():
    g = random_graph(60, 0.08, 9)
    u = 6.0
    k = oracle.k_from_perplexity(u)
    nbr, hop, cnt = oracle.partial_bfs(g.row_ptr, g.col, k)
    beta, pc, conv = oracle.calibrate(hop, cnt, u)
    P_row, P_col, P_val = oracle.symmetrize(nbr, cnt, pc)
    n = g.n
    C = np.zeros((n, n))
    for i in range(n):
        C[i, nbr[i, :cnt[i]]] = pc[i, :cnt[i]]
    Pd = (C + C.T) / (2 * n)
    got = np.zeros((n, n))
    for i in range(n):
        cols = P_col[P_row[i]:P_row[i + 1]]
        assert np.all(np.diff(cols) > 0)
        got[i, cols] = P_val[P_row[i]:P_row[i + 1]]
    assert np.array_equal(got > 0, Pd > 0)
    np.testing.assert_allclose(got, Pd, rtol=1e-15, atol=0)
    assert np.array_equal(got, got.T)
    # each non-empty conditional row contributes 2 * 1/(2n) to the total
    assert abs(P_val.sum() - np.count_nonzero(cnt) / n) < 1e-12


def test_preprocess_grid32_invariants():
    g = synth.grid2d(32, 32)
    aff = oracle.preprocess(g.row_ptr, g.col, 30.0)
    assert aff.nbr.shape == (1024, 90) and np.all(aff.cnt == 90)
    assert np.all(aff.converged == 1)
    assert abs(aff.P_val64.sum() - 1.0) < 1e-12
    assert np.all(aff.P_val64 > 0)
    n = g.n
    dense = csr_matrix((aff.P_val64, aff.P_col, aff.P_row), shape=(n, n)).toarray()
    assert np.array_equal(dense, dense.T)
    assert np.array_equal(aff.P_val32, aff.P_val32)  # FP32 rounding is symmetric too
    d32 = csr_matrix((aff.P_val32, aff.P_col, aff.P_row), shape=(n, n)).toarray()
    assert np.array_equal(d32, d32.T)
