"""Parity of the GPU quality metrics (Sec. 4: NP with r = 2, stress) against
the oracle, through the C ABI.

NP: the per-vertex ball sizes b and intersections c are integers decided in
the same FP32 arithmetic on both sides, so they must match bit for bit; NP
itself is their FP64 mean (summation order differs: 1e-12 relative).
Stress: FP64 sums of the same terms in another order: 1e-12 relative."""
import numpy as np
import pytest

import synth
from oracle import quality

pytestmark = pytest.mark.gpu


def two_components():
    a = synth.grid2d(12, 9)
    b = synth.random_recursive_tree(80, 3)
    u = np.concatenate([np.repeat(np.arange(a.n), np.diff(a.row_ptr)),
                        a.n + np.repeat(np.arange(b.n), np.diff(b.row_ptr))])
    v = np.concatenate([a.col, a.n + b.col])
    return synth.csr_from_edges(a.n + b.n, u, v)


def layouts(g, seed):
    rng = np.random.default_rng(seed)
    yield "gauss", rng.normal(size=(g.n, 2)).astype(np.float32)
    # clustered, with exact duplicates and a wide spread of scales
    Y = (rng.normal(size=(g.n, 2)) * rng.choice([1e-3, 1.0, 30.0], size=(g.n, 1))).astype(np.float32)
    Y[rng.integers(0, g.n, g.n // 10)] = Y[0]
    yield "clustered", Y
    # integer lattice points: many exact distance ties
    yield "lattice", rng.integers(0, 12, size=(g.n, 2)).astype(np.float32)


GRAPHS = {
    "grid": lambda: synth.grid2d(40, 30),
    "sbm": lambda: synth.largest_component(synth.sbm([300, 200, 150], 8.0, 30, 11)),
    "tree": lambda: synth.random_recursive_tree(1500, 5),
    "ba": lambda: synth.barabasi_albert(2000, 3, 8),
    "two": two_components,
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_np_matches_oracle(ltlib, name):
    g = GRAPHS[name]()
    for lname, Y in layouts(g, 7):
        npv, b, c = ltlib.neighbourhood_preservation(g.row_ptr, g.col, Y, return_counts=True)
        npo, bo, co = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
        assert np.array_equal(b.cpu().numpy(), bo), lname
        assert np.array_equal(c.cpu().numpy(), co), lname
        assert npv == pytest.approx(npo, rel=1e-12, abs=1e-15), lname


def test_np_is_one_on_the_lattice(ltlib):
    w, h = 60, 45
    g = synth.grid2d(w, h)
    ids = np.arange(w * h)
    Y = np.stack([ids % w, ids // w], axis=1).astype(np.float32) * 0.25
    npv = ltlib.neighbourhood_preservation(g.row_ptr, g.col, Y)
    assert npv == 1.0


def test_np_hubs_in_the_global_pool(ltlib):
    """A 20,000-vertex Barabasi-Albert graph: the vertices with more than 2048
    two-hop candidates (hubs and their neighbours) go through the hash tables
    in the workspace; per-vertex b and c on all of them and on 300 others
    against the oracle, and a workspace too small for the largest table
    reported as LTSNET_ERR_WORKSPACE."""
    g = synth.barabasi_albert(20000, 4, 3)
    Y = np.random.default_rng(1).normal(size=(g.n, 2)).astype(np.float32)
    npv, b, c = ltlib.neighbourhood_preservation(g.row_ptr, g.col, Y, return_counts=True)
    b, c = b.cpu().numpy(), c.cpu().numpy()
    deg = np.diff(g.row_ptr)
    cand = deg + np.add.reduceat(deg[g.col], g.row_ptr[:-1]) * (deg > 0)
    big = np.flatnonzero(cand > 2048)
    assert big.shape[0] > 20
    rng = np.random.default_rng(4)
    picks = np.concatenate([big, rng.choice(np.flatnonzero(cand <= 2048), 300, replace=False)])
    for v in picks:
        ball = quality.two_hop_ball(g.row_ptr, g.col, int(v))
        assert b[v] == ball.shape[0], v
        near = quality.nearest_in_drawing(Y, int(v), int(b[v]))
        assert c[v] == np.intersect1d(ball, near).shape[0], v
    assert np.all(b > 0)
    assert np.isclose(npv, np.mean(c / (2 * b - c)), rtol=1e-12)
    # the pool is the workspace beyond its fixed part: half the largest table
    # short of it is too small
    def pow2_slots(x):
        s = 4096
        while s < 2 * x:
            s *= 2
        return s

    need = ltlib.lib().ltsnet_quality_workspace_size(g.n, g.col.shape[0])
    fixed = need - 4 * pow2_slots(g.n + g.col.shape[0])
    small = ltlib._workspace(fixed + 4 * pow2_slots(int(cand.max())) // 2)
    with pytest.raises(ltlib.LtsnetError) as e:
        ltlib.neighbourhood_preservation(g.row_ptr, g.col, Y, ws=small)
    assert e.value.code == -2


def test_np_rgg_full_size_sampled(ltlib):
    """The 1M-vertex RGG drawn by the library's Pivot MDS (a drawing that
    keeps graph neighbourhoods close): per-vertex b and c on 150 sampled
    vertices against the oracle's brute force over all n points."""
    g = synth.config_graph("rgg1m")
    Y, _, _ = ltlib.pivot_mds(g.row_ptr, g.col, 30)
    Y = Y.cpu().numpy()
    npv, b, c = ltlib.neighbourhood_preservation(g.row_ptr, g.col, Y, return_counts=True)
    b, c = b.cpu().numpy(), c.cpu().numpy()
    rng = np.random.default_rng(5)
    for v in rng.choice(g.n, 150, replace=False):
        ball = quality.two_hop_ball(g.row_ptr, g.col, int(v))
        assert b[v] == ball.shape[0]
        near = quality.nearest_in_drawing(Y, int(v), int(b[v]))
        assert c[v] == np.intersect1d(ball, near).shape[0]
    assert np.isclose(npv, np.mean(c[b > 0] / (2 * b[b > 0] - c[b > 0])), rtol=1e-12)
    assert 0.0 < npv < 1.0


@pytest.mark.parametrize("name", ["grid", "sbm", "tree", "two"])
def test_stress_matches_oracle(ltlib, name):
    g = GRAPHS[name]()
    Y = np.random.default_rng(3).normal(size=(g.n, 2)).astype(np.float32)
    got = ltlib.stress(g.row_ptr, g.col, Y)
    want = quality.stress(g.row_ptr, g.col, Y.astype(np.float64))
    assert got[2] == want[2] and got[3] == want[3]
    assert got[0] == pytest.approx(want[0], rel=1e-12)
    assert got[1] == pytest.approx(want[1], rel=1e-12)


def test_stress_sampled_sources_and_path(ltlib):
    g = synth.rgg(20000, 8.0, 7)
    Y = np.random.default_rng(4).normal(size=(g.n, 2)).astype(np.float32)
    src = np.random.default_rng(5).choice(g.n, 50, replace=False).astype(np.int32)
    got = ltlib.stress(g.row_ptr, g.col, Y, sources=src)
    want = quality.stress(g.row_ptr, g.col, Y.astype(np.float64), sources=src)
    assert got[2] == want[2] and got[3] == want[3]
    assert got[0] == pytest.approx(want[0], rel=1e-12)
    # a path on an equally spaced line has zero stress at scale 1/spacing
    i = np.arange(499)
    p = synth.csr_from_edges(500, i, i + 1)
    Yp = np.stack([np.arange(500) * 0.5, np.zeros(500)], axis=1).astype(np.float32)
    st, alpha, cnt, skipped = ltlib.stress(p.row_ptr, p.col, Yp)
    assert abs(st) < 1e-13 and alpha == pytest.approx(2.0, rel=1e-12) and cnt == 500 * 499


def test_quality_argument_errors(ltlib):
    g = synth.grid2d(5, 5)
    Y = np.zeros((25, 2), np.float32)
    with pytest.raises(ltlib.LtsnetError) as e:
        ltlib.stress(g.row_ptr, g.col, Y, sources=np.array([3, 25], np.int32))
    assert e.value.code == -1
    col = g.col.copy()
    col[5] = 99
    with pytest.raises(ltlib.LtsnetError) as e:
        ltlib.neighbourhood_preservation(g.row_ptr, col, Y)
    assert e.value.code == -6


def test_quality_degenerate_graphs(ltlib):
    """Two vertices; isolated vertices (an empty ball is skipped by NP; their
    pairs are skipped by stress); a single source."""
    g = synth.csr_from_edges(2, np.array([0]), np.array([1]))
    Y = np.array([[0, 0], [2, 1]], np.float32)
    npv, b, c = ltlib.neighbourhood_preservation(g.row_ptr, g.col, Y, return_counts=True)
    assert npv == 1.0 and list(b.cpu().numpy()) == [1, 1]
    st, alpha, cnt, skipped = ltlib.stress(g.row_ptr, g.col, Y)
    assert abs(st) < 1e-15 and cnt == 2 and skipped == 0
    u = np.arange(5)
    g = synth.csr_from_edges(9, u, u + 1)  # path 0..5, vertices 6, 7, 8 isolated
    Y = np.random.default_rng(1).normal(size=(9, 2)).astype(np.float32)
    npv, b, c = ltlib.neighbourhood_preservation(g.row_ptr, g.col, Y, return_counts=True)
    npo, bo, co = quality.neighbourhood_preservation(g.row_ptr, g.col, Y)
    assert np.array_equal(b.cpu().numpy(), bo) and np.array_equal(c.cpu().numpy(), co)
    assert list(bo[6:]) == [0, 0, 0] and npv == pytest.approx(npo, rel=1e-12)
    got = ltlib.stress(g.row_ptr, g.col, Y, sources=np.array([7], np.int32))
    assert got[2] == 0 and got[3] == 8 and got[0] == 0.0
