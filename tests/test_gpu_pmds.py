"""Parity of the GPU Pivot MDS initial layout (first step of Alg. 1-3)
against the oracle, through the C ABI.

Pivots and BFS distance rows are integers and must match bit for bit.  The
layout is FP32 from FP64 arithmetic: the tolerance is a relative L2 error of
2e-6 per axis (FP32 rounding of each coordinate is 6e-8; the FP64 sums differ
from the oracle's by rounding order and by the eigen-solver's 1e-13 residual,
amplified by 1 / (relative eigen-gap) where the two leading eigenvalues are
close).  Where the gap is below 1e-4 the axes are not unique, and the test
compares pairwise distances, which are."""
import numpy as np
import pytest

import synth
from oracle import pmds

pytestmark = pytest.mark.gpu

Y_TOL = 2e-6


def path(n):
    i = np.arange(n - 1)
    return synth.csr_from_edges(n, i, i + 1)


def two_components():
    a = synth.grid2d(9, 7)
    b = synth.random_recursive_tree(50, 3)
    u = np.concatenate([np.repeat(np.arange(a.n), np.diff(a.row_ptr)),
                        a.n + np.repeat(np.arange(b.n), np.diff(b.row_ptr))])
    v = np.concatenate([a.col, a.n + b.col])
    return synth.csr_from_edges(a.n + b.n, u, v)


def graphs():
    return {
        "grid32": synth.grid2d(32, 32),
        "sbm": synth.largest_component(synth.sbm([400, 300, 200, 100], 8.0, 40, 11)),
        "tree": synth.random_recursive_tree(2000, 5),
        "ba": synth.barabasi_albert(5000, 3, 8),
        "rgg": synth.rgg(20000, 8.0, 7),
        "two_components": two_components(),
    }


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_layout(Y, Yo, lam):
    Y = Y.astype(np.float64)
    gap = (lam[0] - lam[1]) / lam[0] if lam[0] > 0 else 1.0
    if gap > 1e-4:
        for d in range(2):
            if np.any(Yo[:, d] != 0):
                assert rel(Y[:, d], Yo[:, d]) < Y_TOL / min(1.0, gap * 1e2), (d, rel(Y[:, d], Yo[:, d]), gap)
            else:
                assert np.all(Y[:, d] == 0)
    rng = np.random.default_rng(0)
    i = rng.integers(0, Y.shape[0], 4000)
    j = rng.integers(0, Y.shape[0], 4000)
    dg = np.linalg.norm(Y[i] - Y[j], axis=1)
    do = np.linalg.norm(Yo[i] - Yo[j], axis=1)
    assert rel(dg, do) < Y_TOL


def run_both(lt, g, k, first):
    Y, piv, eig, dist = lt.pivot_mds(g.row_ptr, g.col, k, first=first, init_std=1e-4, return_dist=True)
    Yo, po, Do, lam = pmds.pivot_mds(g.row_ptr, g.col, k, first=first, init_std=1e-4)
    return (Y.cpu().numpy(), piv.cpu().numpy(), np.array(eig), dist.cpu().numpy()), (Yo, po, Do, lam)


@pytest.mark.parametrize("name,k,first", [("grid32", 16, 0), ("sbm", 24, 5), ("tree", 10, 1), ("ba", 50, 0),
                                          ("rgg", 40, 123), ("two_components", 8, 70)])
def test_pivot_mds_matches_oracle(ltlib, name, k, first):
    g = graphs()[name]
    (Y, piv, eig, dist), (Yo, po, Do, lam) = run_both(ltlib, g, k, first)
    assert np.array_equal(piv, po)
    want = np.where(Do < 0, 0xFFFF, Do).astype(np.uint16)
    assert np.array_equal(dist.view(np.uint16), want)
    assert np.allclose(eig, lam, rtol=1e-9, atol=1e-12 * lam[0])
    check_layout(Y, Yo, lam)


def test_path_is_a_line(ltlib):
    g = path(3000)
    Y, piv, eig = ltlib.pivot_mds(g.row_ptr, g.col, 7, first=11)
    Y = Y.cpu().numpy().astype(np.float64)
    assert np.all(Y[:, 1] == 0)
    c = np.arange(g.n) - (g.n - 1) / 2
    f = 1e-4 * np.sqrt(2 * g.n / (c * c).sum())
    assert rel(np.abs(Y[:, 0]), np.abs(c) * f) < Y_TOL
    assert eig[1] <= 1e-10 * eig[0]


def test_two_pivots_give_one_axis(ltlib):
    g = graphs()["sbm"]
    (Y, piv, eig, dist), (Yo, po, Do, lam) = run_both(ltlib, g, 2, 0)
    assert np.array_equal(piv, po)
    assert np.all(Y[:, 1] == 0) and np.all(Yo[:, 1] == 0)
    assert rel(Y[:, 0].astype(np.float64), Yo[:, 0]) < Y_TOL


def test_every_vertex_a_pivot(ltlib):
    g = synth.grid2d(9, 6)
    (Y, piv, eig, dist), (Yo, po, Do, lam) = run_both(ltlib, g, g.n, 0)
    assert sorted(piv.tolist()) == list(range(g.n))
    assert np.array_equal(piv, po)
    check_layout(Y, Yo, lam)


def test_deterministic(ltlib):
    g = graphs()["ba"]
    a = ltlib.pivot_mds(g.row_ptr, g.col, 30)[0].cpu().numpy()
    b = ltlib.pivot_mds(g.row_ptr, g.col, 30)[0].cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_argument_errors(ltlib):
    g = synth.grid2d(5, 5)
    for k, first in [(1, 0), (26, 0), (513, 0), (4, -1), (4, 25)]:
        with pytest.raises(ltlib.LtsnetError) as e:
            ltlib.pivot_mds(g.row_ptr, g.col, k, first=first, ws=ltlib._workspace(1 << 20))
        assert e.value.code == -1


def test_bad_column_is_reported(ltlib):
    g = synth.grid2d(20, 20)
    col = g.col.copy()
    col[37] = g.n + 5  # out of range: skipped by the BFS and reported
    with pytest.raises(ltlib.LtsnetError) as e:
        ltlib.pivot_mds(g.row_ptr, col, 4)
    assert e.value.code == -6


def test_distance_above_uint16_is_rejected(ltlib):
    g = path(70000)
    with pytest.raises(ltlib.LtsnetError) as e:
        ltlib.pivot_mds(g.row_ptr, g.col, 3)
    assert e.value.code == -1


def test_rgg1m_hundred_pivots(ltlib):
    """The 1M-vertex random geometric graph with 100 pivots: every pivot and
    every distance row bit-exact; the layout on all n vertices."""
    g = synth.config_graph("rgg1m")
    k = 100
    (Y, piv, eig, dist), (Yo, po, Do, lam) = run_both(ltlib, g, k, 0)
    assert np.array_equal(piv, po)
    assert np.array_equal(dist.view(np.uint16), Do.astype(np.uint16))
    assert np.allclose(eig, lam, rtol=1e-9)
    check_layout(Y, Yo, lam)


def test_two_vertices(ltlib):
    g = synth.csr_from_edges(2, np.array([0]), np.array([1]))
    Y, piv, eig = ltlib.pivot_mds(g.row_ptr, g.col, 2, first=1)
    Y = Y.cpu().numpy().astype(np.float64)
    assert list(piv.cpu().numpy()) == [1, 0]
    # a path of two: x = +-c, and the RMS distance from the centroid is
    # sqrt(2) init_std, so |x| = sqrt(2) 1e-4
    assert np.all(Y[:, 1] == 0) and abs(Y[0, 0] + Y[1, 0]) < 1e-10
    assert abs(abs(Y[0, 0]) - np.sqrt(2) * 1e-4) < 1e-10
