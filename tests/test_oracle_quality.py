"""Pins of the quality-metric oracle (Sec. 4: neighbourhood preservation with
r = 2, and stress) to facts outside it: layouts that preserve every
neighbourhood exactly, scipy's shortest paths and KD-tree neighbours, closed
forms for stress on small graphs, and a numerical minimisation of stress over
the layout scale."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import dijkstra
from scipy.spatial import cKDTree

import synth
from oracle import quality


def path(n):
    i = np.arange(n - 1)
    return synth.csr_from_edges(n, i, i + 1)


def cycle(n):
    i = np.arange(n)
    return synth.csr_from_edges(n, i, (i + 1) % n)


def star(leaves):
    return synth.csr_from_edges(leaves + 1, np.zeros(leaves, np.int64), 1 + np.arange(leaves))


def test_np_is_one_for_a_path_on_a_line():
    g = path(40)
    Y = np.stack([np.arange(40) * 0.37, np.zeros(40)], axis=1).astype(np.float32)
    npv, b, c = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
    assert npv == 1.0
    assert b[0] == 2 and b[1] == 3 and b[20] == 4 and np.array_equal(b, c)


def test_np_is_one_for_a_grid_on_its_lattice():
    """Within two hops on the lattice = within Euclidean distance 2 of it
    (distances 1, sqrt 2 and 2), for interior, edge and corner vertices."""
    w, h = 11, 7
    g = synth.grid2d(w, h)
    ids = np.arange(w * h)
    Y = np.stack([ids % w, ids // w], axis=1).astype(np.float32) * 1.5
    npv, b, c = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
    assert npv == 1.0
    assert b[w + 1 + 2 * w + 2] == 12 and b[0] == 5


@pytest.mark.parametrize("seed", range(4))
def test_np_against_scipy(seed):
    rng = np.random.default_rng(seed)
    n = 300
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < 0.012
    g = synth.csr_from_edges(n, iu[keep], ju[keep])
    Y = rng.normal(size=(n, 2)).astype(np.float32)
    npv, b, c = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
    A = csr_matrix((np.ones(g.col.shape[0]), g.col, g.row_ptr), shape=(n, n))
    D = dijkstra(A, unweighted=True, limit=2.5)
    tree = cKDTree(Y.astype(np.float64))
    scores = []
    for v in range(n):
        ball = set(np.flatnonzero(np.isfinite(D[v])).tolist()) - {v}
        assert b[v] == len(ball)
        if not ball:
            continue
        _, nn = tree.query(Y[v].astype(np.float64), k=len(ball) + 1)
        near = set(np.atleast_1d(nn).tolist()) - {v}
        near = set(list(near)[:len(ball)]) if len(near) > len(ball) else near
        inter = len(ball & near)
        assert c[v] == inter
        scores.append(inter / (2 * len(ball) - inter))
    assert npv == pytest.approx(np.mean(scores), rel=1e-15)


def test_np_counts_hubs():
    """A star with 3000 leaves: every vertex reaches all others within two
    hops (the hub has 6000 two-hop candidates, each leaf 3001), so N_D is all
    other vertices whatever the drawing and NP = 1 -- hubs included."""
    g = star(3000)
    for Y in (np.zeros((3001, 2), np.float32), np.random.default_rng(1).normal(size=(3001, 2)).astype(np.float32)):
        npv, b, c = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
        assert np.all(b == 3000) and np.all(c == 3000) and npv == 1.0
        assert quality.candidate_count(g.row_ptr, g.col, 0) == 6000


def test_np_against_scipy_with_hubs():
    """A Barabasi-Albert graph (hubs of more than 2048 two-hop candidates)
    against scipy's shortest paths and KD-tree neighbours."""
    g = synth.barabasi_albert(3000, 4, seed=3)
    n = g.n
    assert max(quality.candidate_count(g.row_ptr, g.col, v) for v in range(n)) > 2048
    Y = np.random.default_rng(2).normal(size=(n, 2)).astype(np.float32)
    npv, b, c = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
    A = csr_matrix((np.ones(g.col.shape[0]), g.col, g.row_ptr), shape=(n, n))
    D = dijkstra(A, unweighted=True, limit=2.5)
    tree = cKDTree(Y.astype(np.float64))
    scores = []
    for v in range(n):
        ball = set(np.flatnonzero(np.isfinite(D[v])).tolist()) - {v}
        assert b[v] == len(ball)
        _, nn = tree.query(Y[v].astype(np.float64), k=len(ball) + 1)
        near = set(np.atleast_1d(nn).tolist()) - {v}
        near = set(list(near)[:len(ball)]) if len(near) > len(ball) else near
        inter = len(ball & near)
        assert c[v] == inter
        scores.append(inter / (2 * len(ball) - inter))
    assert npv == pytest.approx(np.mean(scores), rel=1e-15)


def test_np_ties_go_to_the_smaller_id():
    # path 0-1-2-3-4 with 3 and 4 placed at the same point: for vertex 0 the
    # ball is {1, 2}; 1 is nearest, then 3 and 4 tie at the next distance
    # with 2 further away, so N_D = {1, 3}
    g = path(5)
    Y = np.array([[0, 0], [1, 0], [5, 0], [2, 0], [2, 0]], np.float32)
    _, b, c = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
    assert b[0] == 2 and c[0] == 1
    assert list(quality.nearest_in_drawing(Y, 0, 3)) == [1, 3, 4]


def test_stress_zero_for_a_path_on_a_line():
    g = path(25)
    for s in (1.0, 0.3, 17.0):
        Y = np.stack([np.arange(25) * s, np.zeros(25)], axis=1)
        st, alpha, cnt, skipped = quality.stress(g.row_ptr, g.col, Y)
        assert abs(st) < 1e-14 and alpha == pytest.approx(1.0 / s, rel=1e-13)
        assert cnt == 25 * 24 and skipped == 0


def test_stress_closed_forms():
    # triangle as an equilateral triangle of side 2: every r = 2
    g = cycle(3)
    Y = np.array([[0, 0], [2, 0], [1, math.sqrt(3)]])
    st, alpha, _, _ = quality.stress(g.row_ptr, g.col, Y)
    assert abs(st) < 1e-15 and alpha == pytest.approx(0.5, rel=1e-15)
    # 4-cycle on the unit square: 8 ordered pairs with r = 1, 4 with r = sqrt(2)/2
    g = cycle(4)
    Y = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
    st, alpha, cnt, _ = quality.stress(g.row_ptr, g.col, Y)
    s1, s2 = 8 + 4 * math.sqrt(2) / 2, 8 + 4 * 0.5
    assert cnt == 12
    assert st == pytest.approx(1 - s1 * s1 / (12 * s2), rel=1e-14)
    assert alpha == pytest.approx(s1 / s2, rel=1e-14)


def test_stress_alpha_minimises_the_literal_formula():
    g = synth.random_recursive_tree(60, 4)
    Y = np.random.default_rng(3).normal(size=(60, 2))
    st, alpha, cnt, _ = quality.stress(g.row_ptr, g.col, Y)
    A = csr_matrix((np.ones(g.col.shape[0]), g.col, g.row_ptr), shape=(60, 60))
    D = dijkstra(A, unweighted=True)
    G = np.sqrt(((Y[:, None] - Y[None]) ** 2).sum(-1))
    off = ~np.eye(60, dtype=bool)

    def literal(a):
        return float((((D[off] - a * G[off]) / D[off]) ** 2).sum() / (60 * 59))

    res = minimize_scalar(literal, bounds=(1e-6, 100), method="bounded", options={"xatol": 1e-12})
    assert res.x == pytest.approx(alpha, rel=1e-6)
    assert literal(alpha) == pytest.approx(st, rel=1e-12)


def test_stress_sources_and_components():
    a, b = path(5), path(4)
    u = np.concatenate([np.arange(4), 5 + np.arange(3)])
    g = synth.csr_from_edges(9, u, u + 1)
    Y = np.random.default_rng(2).normal(size=(9, 2))
    st, alpha, cnt, skipped = quality.stress(g.row_ptr, g.col, Y, sources=[0, 6])
    assert cnt == 4 + 3 and skipped == 4 + 5
    # literal sum over the same pairs
    r = []
    for s, js in ((0, range(1, 5)), (6, (5, 7, 8))):
        for j in js:
            r.append(np.linalg.norm(Y[s] - Y[j]) / abs(s - j))
    r = np.array(r)
    assert st == pytest.approx(1 - r.sum() ** 2 / (len(r) * (r * r).sum()), rel=1e-13)
