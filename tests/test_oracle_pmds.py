"""Pins of the Pivot MDS oracle (the initial layout of Alg. 1-3, Brandes and
Pich's method) to facts outside it: Floyd-Warshall distances, brute-force
max-min choices, closed forms on paths, exact recovery of Euclidean point sets
by classical MDS, and classical MDS of the full graph-distance matrix through
an n x n eigendecomposition."""
import numpy as np
import pytest

import synth
from oracle import pmds


def random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    return synth.csr_from_edges(n, iu[keep], ju[keep])


def path(n):
    i = np.arange(n - 1)
    return synth.csr_from_edges(n, i, i + 1)


def floyd_warshall(g):
    n = g.n
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    for i in range(n):
        D[i, g.col[g.row_ptr[i]:g.row_ptr[i + 1]]] = 1
    for m in range(n):
        D = np.minimum(D, D[:, m:m + 1] + D[m:m + 1, :])
    return D


def pairwise(Y):
    return np.sqrt(((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1))


@pytest.mark.parametrize("seed", range(8))
def test_bfs_distances_match_floyd_warshall(seed):
    # p chosen so that some graphs are disconnected
    g = random_graph(40, 0.05 + 0.01 * seed, 700 + seed)
    FW = floyd_warshall(g)
    for s in range(0, g.n, 7):
        d = pmds.bfs_distances(g.row_ptr, g.col, s)
        want = np.where(np.isinf(FW[s]), -1, FW[s]).astype(np.int64)
        assert np.array_equal(d, want)


def test_bfs_distances_path_closed_form():
    g = path(50)
    for s in (0, 17, 49):
        assert np.array_equal(pmds.bfs_distances(g.row_ptr, g.col, s), np.abs(np.arange(50) - s))


@pytest.mark.parametrize("seed", range(6))
def test_maxmin_pivots_brute_force(seed):
    g = random_graph(36, 0.06 + 0.02 * seed, 800 + seed)
    FW = floyd_warshall(g)
    k = 12
    piv, D = pmds.maxmin_pivots(g.row_ptr, g.col, k, first=seed)
    assert piv[0] == seed
    for t in range(1, k):
        nearest = FW[piv[:t]].min(axis=0)  # inf where no pivot reaches
        best = nearest.max()
        assert piv[t] == np.flatnonzero(nearest == best)[0]
    for t in range(k):
        want = np.where(np.isinf(FW[piv[t]]), -1, FW[piv[t]])
        assert np.array_equal(D[t], want.astype(np.int64))


def test_maxmin_pivots_path_by_hand():
    g = path(11)
    piv, _ = pmds.maxmin_pivots(g.row_ptr, g.col, 5, first=0)
    # 0; the far end 10; the middle 5; then distance 2 first reached at 2
    assert list(piv[:4]) == [0, 10, 5, 2]


def test_sign_rule_on_an_exact_tie():
    """k = 2 on a path of 9 with pivots 0 and 8: v = +-(1, -1)/sqrt(2), a tie
    in magnitude, and the rule takes the first entry positive.  Then
    C v = -1/2 J_n (a_0 - a_1)/sqrt(2) with a_i0 - a_i1 = i^2 - (8 - i)^2 =
    16 (i - 4), so x_i is proportional to -(i - 4): decreasing along the
    path."""
    g = path(9)
    Y, piv, D, lam = pmds.pivot_mds(g.row_ptr, g.col, 2, first=0, init_std=0.0)
    assert list(piv) == [0, 8]
    assert np.all(np.diff(Y[:, 0]) < 0)
    assert np.all(Y[:, 1] == 0)


def test_disconnected_pivot_goes_to_the_other_component():
    # paths 0..5 and 6..10
    u = np.concatenate([np.arange(5), 6 + np.arange(4)])
    g = synth.csr_from_edges(11, u, u + 1)
    piv, D = pmds.maxmin_pivots(g.row_ptr, g.col, 3, first=2)
    # smallest index of the unreached component, then the far end of the
    # longer reach: 10 is 4 from 6, while 5 is 3 from 2
    assert list(piv) == [2, 6, 10]
    A = pmds.squared_distances(D)
    # largest finite pivot distance is 4, so pairs across components get 5
    assert A[8, 0] == 25 and A[1, 1] == 25 and A[1, 0] == 1


@pytest.mark.parametrize("seed", range(4))
def test_classical_mds_recovers_euclidean_points(seed):
    """All points as pivots and Euclidean squared distances: classical MDS
    returns the point set up to an orthogonal map and a shift, so all pairwise
    distances come back.  A dropped half, a centring over the wrong index or
    another axis scale breaks this."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(30, 2)) * np.array([3.0, 1.0])
    A = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    Y, lam = pmds.pmds_coords(A, init_std=0.0)
    assert np.allclose(pairwise(Y), pairwise(X), rtol=0, atol=1e-9)
    assert lam[0] >= lam[1] > 0


def test_all_vertices_as_pivots_is_classical_mds_of_the_graph():
    """k = n: Pivot MDS is classical MDS of the full hop-distance matrix,
    computed here independently from the n x n double-centred matrix B."""
    g = synth.grid2d(7, 5)
    n = g.n
    piv, D = pmds.maxmin_pivots(g.row_ptr, g.col, n, first=0)
    assert sorted(piv.tolist()) == list(range(n))
    Y, _ = pmds.pmds_coords(pmds.squared_distances(D), init_std=0.0)
    FW = floyd_warshall(g)
    J = np.eye(n) - 1.0 / n
    B = -0.5 * J @ (FW ** 2) @ J
    lam, U = np.linalg.eigh(B)
    top = np.argsort(lam)[::-1][:2]
    X = U[:, top] * np.sqrt(lam[top])
    assert np.allclose(pairwise(Y), pairwise(X), rtol=0, atol=1e-9)


@pytest.mark.parametrize("k", [2, 3, 9])
def test_path_is_laid_out_on_a_line(k):
    """A path's squared distances have rank-one double centring: any pivot
    set gives x proportional to i - (n-1)/2 and a zero second axis."""
    n, std = 21, 1e-4
    g = path(n)
    Y, piv, _, _ = pmds.pivot_mds(g.row_ptr, g.col, k, first=3, init_std=std)
    c = np.arange(n) - (n - 1) / 2
    f = std * np.sqrt(2 * n / (c * c).sum())
    assert np.all(Y[:, 1] == 0)
    assert np.allclose(np.abs(Y[:, 0]), np.abs(c) * f, rtol=1e-9, atol=1e-12 * std)
    assert np.allclose(Y[:, 0], c * f, rtol=1e-9, atol=1e-12 * std) or np.allclose(Y[:, 0], -c * f, rtol=1e-9, atol=1e-12 * std)


@pytest.mark.parametrize("name", ["grid", "sbm", "tree"])
def test_layout_invariants(name):
    """Centroid at the origin (C is centred over the vertices), the two axes
    uncorrelated (C v_1 and C v_2 are orthogonal), RMS spread set by init_std,
    and the sign rule (first entry within a relative 1e-9 of the largest
    magnitude positive; recovered here by least squares, to 1e-6)."""
    if name == "grid":
        g = synth.grid2d(12, 9)
    elif name == "sbm":
        g = synth.largest_component(synth.sbm([60, 40, 30], 6.0, 6, 5))
    else:
        g = synth.random_recursive_tree(150, 9)
    std = 1e-4
    Y, piv, D, lam = pmds.pivot_mds(g.row_ptr, g.col, 10, first=1, init_std=std)
    n = g.n
    assert abs(Y[:, 0].sum()) < 1e-12 * n * std and abs(Y[:, 1].sum()) < 1e-12 * n * std
    assert abs((Y[:, 0] * Y[:, 1]).sum()) < 1e-10 * (Y * Y).sum()
    assert np.isclose(np.sqrt((Y * Y).sum() / (2 * n)), std, rtol=1e-12)
    assert len(set(piv.tolist())) == 10
    # sign rule: x_d = C v_d / sqrt(sigma_d) with v_d's largest entry positive,
    # so v_d is recovered from the layout by least squares on C
    A = pmds.squared_distances(D)
    Jn_A = A - A.mean(axis=0, keepdims=True)
    C = -0.5 * (Jn_A - Jn_A.mean(axis=1, keepdims=True))
    for d in range(2):
        v = np.linalg.lstsq(C, Y[:, d], rcond=None)[0]
        v -= v.mean()  # the null direction 1 of C
        a = np.abs(v)
        j = np.flatnonzero(a >= (1 - 1e-6) * a.max())[0]
        assert v[j] > 0
