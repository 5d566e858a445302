"""Pins of the quadtree oracle (BH-tsNET Alg. 1, FIt-tsNET Alg. 2, Eq. 7) to
facts outside it: theta = 0 gives the exact O(n^2) sums of the C oracle; a
far cluster is summarised as m times the kernel at its mean (closed form);
the error against the exact sums shrinks with theta; the tree partitions the
points and every centre lies in its cell."""
import numpy as np
import pytest

import oracle
from oracle import quadtree


def exact(Y32, eps=quadtree.EPS_DEFAULT):
    n = Y32.shape[0]
    empty = (np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    A, R, E, Z = oracle.exact_sums(Y32.astype(np.float64), *empty, eps=eps)
    return Z, R, E


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("seed", range(3))
def test_theta_zero_is_exact(seed):
    rng = np.random.default_rng(seed)
    Y = (rng.normal(size=(300, 2)) * rng.choice([0.01, 1.0, 20.0], size=(300, 1))).astype(np.float32)
    Y[rng.integers(0, 300, 20)] = Y[5]  # coincident points share depth-16 cells
    Zp, R, E = quadtree.sums(Y, 0.0)
    Z, Rx, Ex = exact(Y)
    assert Zp.sum() == pytest.approx(Z, rel=1e-12)
    assert rel(R, Rx) < 1e-12 and rel(E, Ex) < 1e-12


def test_far_cluster_is_one_summary():
    """A probe at the origin and m points spread over [60, 100]^2: the
    top-right quadrant (width e/2 < 50) holds exactly the cluster and
    passes the test at theta = 0.5 (2500 < 0.25 |c|^2), so the probe sees
    m times the kernel at the cluster's mean.  The centre is rounded to FP32:
    1e-6 relative.  The exact sums differ from the summary by about 2%."""
    rng = np.random.default_rng(4)
    m = 40
    cl = (60.0 + rng.random((m, 2)) * 40.0).astype(np.float32)
    Y = np.vstack([np.zeros((1, 2), np.float32), cl])
    Zp, R, E = quadtree.sums(Y, 0.5)
    mean = cl.astype(np.float64).mean(axis=0)
    d = -mean
    d2 = d @ d
    q = 1.0 / (1.0 + d2)
    assert Zp[0] == pytest.approx(m * q, rel=1e-6)
    assert np.allclose(R[0], m * q * q * d, rtol=1e-6)
    assert np.allclose(E[0], m * d / (quadtree.EPS_DEFAULT + d2), rtol=1e-6)
    Z, Rx, Ex = exact(Y)
    assert abs(R[0, 0] / Rx[0, 0] - 1) > 1e-3


def test_error_shrinks_with_theta():
    rng = np.random.default_rng(7)
    Y = rng.normal(size=(500, 2)).astype(np.float32) * 5
    Z, Rx, Ex = exact(Y)
    errs = []
    for th in (1.0, 0.5, 0.25):
        Zp, R, E = quadtree.sums(Y, th)
        errs.append((rel(R, Rx), rel(E, Ex), abs(Zp.sum() / Z - 1)))
    for k in range(3):
        assert errs[2][k] < errs[1][k] < errs[0][k]
    assert errs[1][0] < 0.05 and errs[1][1] < 0.05


def test_tree_partitions_and_centres():
    rng = np.random.default_rng(8)
    Y = rng.random((400, 2)).astype(np.float32) * np.array([3.0, 1.0], np.float32)
    t = quadtree.Tree(Y)
    sc = t.code[t.order]
    assert np.all(np.diff(sc.astype(np.int64)) >= 0)
    for l in range(quadtree.LEVELS):
        for (a, b) in t.nodes[l]:
            ch = t.children(l, a, b)
            if b - a > 1:
                assert ch[0][0] == a and ch[-1][1] == b
                assert all(ch[k][1] == ch[k + 1][0] for k in range(len(ch) - 1))
                assert 1 <= len(ch) <= 4
            c = t.centre(a, b).astype(np.float64)
            pts = Y[t.order[a:b]].astype(np.float64)
            assert np.all(c >= pts.min(axis=0) - 1e-6) and np.all(c <= pts.max(axis=0) + 1e-6)
            assert np.allclose(c, pts.mean(axis=0), rtol=0, atol=1e-6)


def test_gradient_assembles_like_the_exact_one_at_theta_zero():
    rng = np.random.default_rng(9)
    import synth

    g = synth.grid2d(8, 6)
    aff = oracle.preprocess(g.row_ptr, g.col, 5.0)
    Y = rng.normal(size=(g.n, 2)).astype(np.float32)
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    gq, _ = quadtree.gradient(Y, aff.P_row, aff.P_col, aff.P_val64, st, 0.0)
    ge, _ = oracle.exact_gradient(Y.astype(np.float64), aff.P_row, aff.P_col, aff.P_val64, st)
    assert rel(gq, ge) < 1e-6  # A in the oracle's attraction uses FP32 coordinates


def test_own_cell_is_never_a_summary():
    """theta = 10 accepts almost any node, but not one that holds the point
    itself: of two points at distance 1, each sees the other exactly
    (Zp = 1/2, R = -+(1/4, 0)); summarising the root would give
    2/(1 + 1/4) instead."""
    Y = np.array([[0, 0], [1, 0]], np.float32)
    Zp, R, E = quadtree.sums(Y, 10.0)
    assert np.allclose(Zp, 0.5, rtol=1e-15)
    assert np.allclose(R, [[-0.25, 0], [0.25, 0]], rtol=1e-15)
    assert np.allclose(E, [[-1 / 1.05, 0], [1 / 1.05, 0]], rtol=1e-15)
