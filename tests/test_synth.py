"""The seeded synthetic inputs have the shapes the input recipe states (the
paper's SNAP, GION and SuiteSparse graphs are not used): CSR invariants,
sizes, degrees and determinism of every family, the 1M-vertex RGG's
largest-component size, and the batch's size distribution."""
import math

import numpy as np
import pytest

import synth


def check_csr(g):
    n = g.n
    assert g.row_ptr.dtype == np.int64 and g.col.dtype == np.int32
    assert g.row_ptr[0] == 0 and np.all(np.diff(g.row_ptr) >= 0) and g.row_ptr[-1] == g.col.shape[0]
    assert np.all((g.col >= 0) & (g.col < n))
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    assert not np.any(rows == g.col)  # no self-loops
    for i in range(0, n, max(1, n // 200)):
        c = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)  # sorted, no duplicates
    # both directions stored: the edge multiset is symmetric
    a = rows.astype(np.int64) * n + g.col
    b = g.col.astype(np.int64) * n + rows
    assert np.array_equal(np.sort(a), np.sort(b))


def test_grid_and_tree_closed_forms():
    g = synth.grid2d(32, 32)
    check_csr(g)
    assert g.n == 1024 and g.m == 2 * 32 * 31
    t = synth.random_recursive_tree(5000, 3)
    check_csr(t)
    assert t.m == 4999


def test_families_are_deterministic_and_well_formed():
    for make in (lambda s: synth.sbm([50, 40, 30], 6.0, 10, s), lambda s: synth.rgg(3000, 8.0, s),
                 lambda s: synth.barabasi_albert(3000, 4, s), lambda s: synth.random_recursive_tree(500, s)):
        a, b, c = make(1), make(1), make(2)
        check_csr(a)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
        assert not (a.n == c.n and a.col.shape == c.col.shape and np.array_equal(a.col, c.col))


def test_barabasi_albert_edges():
    g = synth.barabasi_albert(20000, 4, 5)
    check_csr(g)
    # each new vertex brings 4 edges: m = 4 (n - m0) + the seed clique's edges
    assert abs(g.m - 4 * g.n) <= 16
    deg = np.diff(g.row_ptr)
    assert deg.min() >= 4 and deg.max() > 5 * deg.mean()  # heavy tail: hubs


def test_rgg_mean_degree_and_component():
    g = synth.rgg(200_000, 8.0, 3)
    check_csr(g)
    assert 0.98 * 200_000 < g.n <= 200_000  # largest component of a supercritical RGG
    assert abs(2 * g.m / g.n - 8.0) < 0.4


@pytest.mark.slow
def test_rgg1m_workload_size():
    g = synth.config_graph("rgg1m")
    assert g.n == 999_019 and g.m == 3_996_774


def test_initial_layout():
    Y = synth.initial_layout(100_000, 1)
    assert Y.dtype == np.float32 and Y.shape == (100_000, 2)
    assert abs(Y.std() / 1e-4 - 1) < 0.01 and abs(Y.mean()) < 1e-6
    assert np.array_equal(Y, synth.initial_layout(100_000, 1))


def test_graph_batch_sizes():
    gs = synth.graph_batch(512)
    ns = np.array([g.n for g in gs])
    assert len(gs) == 512 and ns.min() >= 150 and ns.max() <= 20_500
    # log-uniform on [200, 20000]: median near sqrt(200 * 20000) = 2000
    assert 1400 < np.median(ns) < 2800
    assert abs(ns.sum() - 2.365e6) < 0.05e6
    for g in gs[:30]:
        check_csr(g)
