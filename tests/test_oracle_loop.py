"""Pins of the oracle's loop terms (Alg. 3 loop body) to independent facts:
central finite differences of the cost (Eq. 1), closed forms for two points,
Newton's third law, polynomial reproduction of the Lagrange spread, the direct
O(M^4) convolution against the FFT one, the transpose identity for Z, and
convergence of the interpolated sums to the exact O(n^2) sums."""
import math

import numpy as np
import pytest

import oracle
import synth


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def small_problem(n=60, seed=0, scale=2.0):
    g = synth.sbm([n // 2, n - n // 2], 6.0, 6, seed=seed)
    aff = oracle.preprocess(g.row_ptr, g.col, 4.0)
    Y = np.random.default_rng(seed).standard_normal((g.n, 2)) * scale
    return g, aff, Y


@pytest.mark.parametrize("lam", [(1.0, 1.2, 0.0, 1.0), (1.0, 0.01, 0.6, 1.0), (0.5, 0.3, 2.0, 1.0)])
def test_exact_gradient_central_differences(lam):
    """Analytic exact gradient vs central differences of the exact cost on
    every coordinate (n = 60), step 1e-6 * max(1, |x|)."""
    g, aff, Y = small_problem()
    st = oracle.Stage(1, *lam, 0.5)
    grad, _ = oracle.exact_gradient(Y, aff.P_row, aff.P_col, aff.P_val64, st)
    fd = np.zeros_like(Y)
    for i in range(Y.shape[0]):
        for d in range(2):
            h = 1e-6 * max(1.0, abs(Y[i, d]))
            Yp = Y.copy(); Yp[i, d] += h
            Ym = Y.copy(); Ym[i, d] -= h
            fd[i, d] = (oracle.exact_cost(Yp, aff.P_row, aff.P_col, aff.P_val64, st)[0]
                        - oracle.exact_cost(Ym, aff.P_row, aff.P_col, aff.P_val64, st)[0]) / (2 * h)
    assert rel(grad, fd) < 1e-6


def test_literal_entropy_matches_reading_at_eps0():
    """At eps = 0 the paper's -(l_r/2n^2) sum ln|d| equals the reading's
    -(l_r/4n^2) sum ln(d^2) (Eq. 1 vs the Sec. 3.3 kernel form)."""
    g, aff, Y = small_problem()
    st = oracle.Stage(1, 0.0, 0.0, 1.0, 1.0, 0.5)
    a = oracle.exact_cost(Y, aff.P_row, aff.P_col, aff.P_val64, st, eps=0.0)[0]
    b = oracle.exact_cost(Y, aff.P_row, aff.P_col, aff.P_val64, st, eps=0.0, literal=True)[0]
    assert abs(a - b) <= 1e-12 * abs(a)


def test_two_point_closed_form():
    """Points (+a, 0), (-a, 0), P = [[0, 1/2], [1/2, 0]]: Z = 2/(1+4a^2);
    attraction, repulsion and entropy act along x with closed-form values."""
    a = 0.7
    Y = np.array([[a, 0.0], [-a, 0.0]])
    P_row = np.array([0, 1, 2]); P_col = np.array([1, 0], np.int32); P_val = np.array([0.5, 0.5])
    eps = 0.05
    A, R, E, Z = oracle.exact_sums(Y, P_row, P_col, P_val, eps)
    d2 = 4 * a * a
    assert abs(Z - 2 / (1 + d2)) < 1e-15
    np.testing.assert_allclose(A[0], [0.5 * 2 * a / (1 + d2), 0.0], atol=1e-15)
    np.testing.assert_allclose(R[0], [2 * a / (1 + d2) ** 2, 0.0], atol=1e-15)
    np.testing.assert_allclose(E[0], [2 * a / (eps + d2), 0.0], atol=1e-15)
    np.testing.assert_allclose(A[1], -A[0], atol=1e-15)
    st = oracle.Stage(1, 1.0, 0.3, 0.6, 1.0, 0.5)
    g, _ = oracle.exact_gradient(Y, P_row, P_col, P_val, st, eps)
    gx = 4 * (0.5 * 2 * a / (1 + d2) - (1.0 / Z) * 2 * a / (1 + d2) ** 2) + 0.3 / 2 * a - 0.6 / 4 * 2 * a / (eps + d2)
    assert abs(g[0, 0] - gx) < 1e-14 and abs(g[0, 1]) < 1e-15


def test_newton_third_law():
    """With symmetric P the KL and entropy forces cancel in total; the
    gradient sums to the compression term (l_c/n) sum X."""
    g, aff, Y = small_problem(80, 3)
    st = oracle.Stage(1, 1.0, 0.4, 0.6, 1.0, 0.5)
    grad, parts = oracle.exact_gradient(Y, aff.P_row, aff.P_col, aff.P_val64, st)
    scale = np.abs(parts["R"]).sum()
    assert np.abs(parts["A"].sum(0)).max() < 1e-14 * max(1.0, np.abs(parts["A"]).sum())
    assert np.abs(parts["R"].sum(0)).max() < 1e-13 * scale
    assert np.abs(parts["E"].sum(0)).max() < 1e-13 * np.abs(parts["E"]).sum()
    np.testing.assert_allclose(grad.sum(0), 0.4 / Y.shape[0] * Y.sum(0), atol=1e-12)


def test_grad_pvals_central_differences():
    g, aff, Y = small_problem(40, 5)
    st = oracle.Stage(1, 1.0, 0.0, 0.0, 1.0, 0.5)
    gp = oracle.grad_pvals(Y, aff.P_row, aff.P_col, aff.P_val64, st)
    rng = np.random.default_rng(0)
    pos = np.flatnonzero(aff.P_val64 > 1e-5)  # cost resolution limits the difference quotient
    for e in rng.choice(pos, 20, replace=False):
        h = 1e-4 * aff.P_val64[e]
        vp = aff.P_val64.copy(); vp[e] += h
        vm = aff.P_val64.copy(); vm[e] -= h
        fd = (oracle.exact_cost(Y, aff.P_row, aff.P_col, vp, st)[0]
              - oracle.exact_cost(Y, aff.P_row, aff.P_col, vm, st)[0]) / (2 * h)
        assert abs(fd - gp[e]) < 1e-6 * max(1.0, abs(gp[e]))


@pytest.mark.parametrize("P", [2, 3, 4, 5, 7])
def test_spread_reproduces_polynomials(P):
    """Lagrange interpolation on P nodes reproduces polynomials of degree
    < P, so the spread grid's moments equal the points' moments exactly:
    sum_t W0 = n, sum_t W0 xi_x = sum x~, sum_t W1 = sum x~, ..."""
    rng = np.random.default_rng(P)
    Y = (rng.standard_normal((200, 2)) * 3).astype(np.float32)
    gi = oracle.grid_rule(Y, oracle.GridParams(nodes_per_box=P, min_boxes=5))
    W, box = oracle.spread(Y, gi, P)
    xi = gi.lo + (np.arange(gi.M) + 0.5) * gi.s - gi.centre  # node coordinates, centred
    Yc = Y.astype(np.float64) - gi.centre
    assert abs(W[0].sum() - Y.shape[0]) < 1e-10
    assert abs((W[0] * xi[None, :]).sum() - Yc[:, 0].sum()) < 1e-9
    assert abs((W[0] * xi[:, None]).sum() - Yc[:, 1].sum()) < 1e-9
    assert abs(W[1].sum() - Yc[:, 0].sum()) < 1e-9 and abs(W[2].sum() - Yc[:, 1].sum()) < 1e-9
    assert abs(W[3].sum() - (Yc ** 2).sum()) < 1e-8
    if P >= 3:
        assert abs((W[0] * xi[None, :] ** 2).sum() - (Yc[:, 0] ** 2).sum()) < 1e-8
    # every point's box contains it
    lo, h = np.float32(gi.lo), np.float32(gi.h)
    for d in range(2):
        left = lo + box[:, d].astype(np.float64) * gi.h
        assert np.all(Y[:, d] >= left - 1e-6 * gi.h) and np.all(Y[:, d] <= left + gi.h * (1 + 1e-5))


def test_grid_rule():
    rng = np.random.default_rng(2)
    for scale in (1e-4, 0.3, 7.0, 40.0, 500.0):
        Y = (rng.standard_normal((300, 2)) * scale).astype(np.float32)
        gp = oracle.GridParams()
        gi = oracle.grid_rule(Y, gp)
        ext = np.float32(Y.max()) - np.float32(Y.min())
        assert gi.lo == Y.min() and gi.hi == Y.max()
        assert gi.I >= gp.min_boxes and gi.I <= gp.max_boxes
        v = gi.I
        for f in (2, 3, 5):
            while v % f == 0:
                v //= f
        assert v == 1
        if ext / gp.box_width_max <= gp.max_boxes:
            assert gi.h <= gp.box_width_max * (1 + 1e-6)
        assert gi.M == gi.I * gp.nodes_per_box


def test_grid_rule_by_hand():
    """Hand-computed cases of the grid rule: extent 60.5 at box width 1 gives
    ceil(60.5) = 61 boxes, rounded up to the next 5-smooth size 64 (not 63 =
    7 * 9, not floor 60); h = 60.5 / 64, three nodes per box, the centre at
    the midpoint 27.25.  A cap of 630 (= 2 * 3^2 * 5 * 7) falls back to the
    largest 5-smooth size below it, 625."""
    Y = np.array([[-3.0, 0.0], [57.5, 10.0]], np.float32)
    gi = oracle.grid_rule(Y, oracle.GridParams(box_width_max=1.0, min_boxes=50, max_boxes=640, nodes_per_box=3))
    assert (gi.lo, gi.hi, gi.ext, gi.I, gi.M) == (-3.0, 57.5, 60.5, 64, 192)
    assert gi.h == float(np.float32(60.5) / np.float32(64)) and gi.centre == 27.25
    assert gi.s == float(np.float32(gi.h) / np.float32(3))
    Y = np.array([[0.0, 0.0], [900.0, 1.0]], np.float32)
    gi = oracle.grid_rule(Y, oracle.GridParams(box_width_max=1.0, min_boxes=50, max_boxes=630, nodes_per_box=2))
    assert gi.I == 625 and gi.M == 1250


def test_direct_and_fft_convolution_agree():
    rng = np.random.default_rng(7)
    for M, s in ((9, 0.3), (24, 0.11), (30, 1.7)):
        W = rng.standard_normal((4, M, M))
        a = oracle.conv_direct(W, s, 0.05)
        b = oracle.conv_fft(W, s, 0.05)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_z_grid_form_equals_point_form():
    g, aff, Y = small_problem(120, 8, 5.0)
    Y32 = Y.astype(np.float32)
    Phi, W, fld, gi = oracle.interp_fields(Y32, oracle.GridParams(min_boxes=10))
    a = oracle.z_from_points(Y32, Phi, gi.centre)
    b = oracle.z_from_grid(W, fld, Y32.shape[0])
    assert abs(a - b) <= 1e-12 * abs(a)


def test_interp_exact_when_grid_is_fine():
    """At an extent far below the kernels' widths, interpolation is exact to
    rounding (init layout N(0, 1e-4^2))."""
    g = synth.grid2d(16, 16)
    aff = oracle.preprocess(g.row_ptr, g.col, 10.0)
    Y = synth.initial_layout(g.n, 1)
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    ge, pe = oracle.exact_gradient(Y.astype(np.float64), aff.P_row, aff.P_col, aff.P_val64, st)
    gi, pi = oracle.interp_gradient(Y, aff.P_row, aff.P_col, aff.P_val64, st, oracle.GridParams())
    assert rel(gi, ge) < 1e-9 and rel(pi["R"], pe["R"]) < 1e-9 and rel(pi["E"], pe["E"]) < 1e-9
    assert abs(pi["Z"] - pe["Z"]) / pe["Z"] < 1e-10


def test_interp_converges_to_exact():
    """Interpolated sums approach the exact sums as nodes per box grow and as
    boxes shrink (monotone in both)."""
    g, aff, Y = small_problem(300, 11, 6.0)
    Y32 = Y.astype(np.float32)
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    ge, pe = oracle.exact_gradient(Y32.astype(np.float64), aff.P_row, aff.P_col, aff.P_val64, st)
    errs = {}
    for P in (3, 5, 7):
        for h in (1.0, 0.5, 0.25):
            gp = oracle.GridParams(nodes_per_box=P, box_width_max=h, min_boxes=1)
            _, pi = oracle.interp_gradient(Y32, aff.P_row, aff.P_col, aff.P_val64, st, gp)
            errs[P, h] = (rel(pi["R"], pe["R"]), rel(pi["E"], pe["E"]))
    for P in (3, 5, 7):
        assert errs[P, 1.0][0] > errs[P, 0.5][0] > errs[P, 0.25][0]
        assert errs[P, 0.5][1] > errs[P, 0.25][1]
    for h in (0.5, 0.25):
        assert errs[3, h][0] > errs[5, h][0] > errs[7, h][0]
        assert errs[3, h][1] > errs[5, h][1] > errs[7, h][1]
    assert errs[7, 0.25][0] < 1e-7 and errs[7, 0.25][1] < 1e-5


def test_update_rule():
    """Gains grow by 0.2 where the gradient's sign differs from the last
    step's, shrink by x0.8 elsewhere, floor 0.01; momentum step."""
    Y = np.zeros((3, 2)); upd = np.array([[1.0, -1.0], [0.0, 2.0], [-3.0, 0.0]])
    gains = np.array([[1.0, 0.011], [1.0, 1.0], [0.5, 0.5]])
    grad = np.array([[1.0, -1.0], [1.0, -1.0], [2.0, 0.0]])
    Y2, u2, g2 = oracle.update(Y, upd, gains, grad, 0.5, 10.0)
    np.testing.assert_allclose(g2, [[0.8, 0.01], [1.2, 1.2], [0.7, 0.4]])
    np.testing.assert_allclose(u2, 0.5 * upd - 10.0 * g2 * grad)
    np.testing.assert_allclose(Y2, u2)


def test_log_kernel_sum_fft_equals_direct():
    """The entropy double sum on the grid: FFT embedding equals the direct
    sum over node pairs."""
    rng = np.random.default_rng(11)
    W0 = rng.random((9, 9))
    W0[rng.random((9, 9)) < 0.3] = 0.0
    a = oracle.log_kernel_sum(W0, 0.37, 0.05)
    b = oracle.log_kernel_sum_direct(W0, 0.37, 0.05)
    assert abs(a - b) <= 1e-11 * abs(b)


def test_interp_entropy_sum_converges_to_exact():
    """sum_{i,j} ln(eps + d^2) interpolated on finer and finer grids
    approaches the exact double sum (self terms n ln eps included), with the
    error falling as the boxes shrink."""
    rng = np.random.default_rng(5)
    n = 40
    Y = (rng.standard_normal((n, 2)) * 1.5).astype(np.float32)
    P_row = np.zeros(n + 1, np.int64)
    P_col = np.zeros(0, np.int32)
    P_val = np.zeros(0, np.float64)
    _, parts = oracle.exact_cost(Y.astype(np.float64), P_row, P_col, P_val, oracle.Stage(1, 0, 0, 1, 1, 0))
    exact = -parts["ent"] * 4 * n * n + n * np.log(oracle.EPS_DEFAULT)  # sum over all ordered pairs incl. i = j
    errs = []
    for bw in (1.0, 0.25, 0.0625):
        gp = oracle.GridParams(box_width_max=bw, min_boxes=4, max_boxes=1350)
        gi = oracle.grid_rule(Y, gp)
        W, _ = oracle.spread(Y, gi, gp.nodes_per_box)
        errs.append(abs(oracle.log_kernel_sum(W[0], gi.s, gp.eps) - exact) / abs(exact))
    assert errs[2] < errs[0] and errs[2] < 1e-4, errs


def test_exact_gradient_with_unnormalised_P():
    """P scaled by 3 (S = 3): the repulsion carries S / Z, and the gradient
    still matches central differences of the cost (whose KL term has
    S ln Z)."""
    g, aff, Y = small_problem()
    st = oracle.Stage(1, 1.0, 0.05, 0.3, 1.0, 0.5)
    pv = aff.P_val64 * 3.0
    grad, parts = oracle.exact_gradient(Y, aff.P_row, aff.P_col, pv, st)
    assert abs(parts["S"] - 3.0) < 1e-12
    fd = np.zeros_like(Y)
    for i in range(Y.shape[0]):
        for d in range(2):
            h = 1e-6 * max(1.0, abs(Y[i, d]))
            Yp = Y.copy(); Yp[i, d] += h
            Ym = Y.copy(); Ym[i, d] -= h
            fd[i, d] = (oracle.exact_cost(Yp, aff.P_row, aff.P_col, pv, st)[0]
                        - oracle.exact_cost(Ym, aff.P_row, aff.P_col, pv, st)[0]) / (2 * h)
    assert rel(grad, fd) < 1e-6


def test_interp_cost_entropy_converges_to_exact():
    """The cost's entropy term from the grid (the double sum minus the n self
    terms ln eps) approaches the exact term on a fine grid; keeping the self
    terms would be off by lambda_r ln(eps) / (4n)."""
    rng = np.random.default_rng(6)
    n = 40
    Y = (rng.standard_normal((n, 2)) * 1.5).astype(np.float32)
    P = (np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float64))
    st = oracle.Stage(1, 0.0, 0.0, 1.0, 1.0, 0.5)
    _, parts = oracle.exact_cost(Y.astype(np.float64), *P, st)
    gp = oracle.GridParams(box_width_max=0.0625, min_boxes=4, max_boxes=1350)
    got = oracle.interp_cost(Y, *P, st, gp)["ent"]
    self_terms = abs(np.log(oracle.EPS_DEFAULT) / (4 * n))
    assert abs(got - parts["ent"]) < 0.05 * self_terms


def test_exact_rows_and_z_equal_the_full_exact_sums():
    """The row-subset exact sums and the stand-alone Z (used for sampled checks
    of large layouts) equal the all-rows pass, which the central differences
    above pin; rows may repeat and come in any order."""
    g, aff, Y = small_problem(n=80, seed=3)
    A, R, E, Z = oracle.exact_sums(Y, aff.P_row, aff.P_col, aff.P_val64)
    rows = np.array([5, 0, 79, 5, 41], np.int32)
    A2, R2, E2 = oracle.exact_rows(Y, aff.P_row, aff.P_col, aff.P_val64, rows)
    assert np.array_equal(A2, A[rows]) and np.array_equal(R2, R[rows]) and np.array_equal(E2, E[rows])
    assert abs(oracle.exact_z(Y) - Z) <= 1e-13 * Z
    with pytest.raises(ValueError):
        oracle.exact_rows(Y, aff.P_row, aff.P_col, aff.P_val64, np.array([80], np.int32))


@pytest.mark.parametrize("lam", [(1.0, 1.2, 0.0, 1.0), (1.0, 0.01, 0.6, 1.0)])
def test_cost_step_equals_differences_of_the_full_cost(lam):
    """The O(n + nnz) central difference of the exact cost equals the
    difference of two full O(n^2) cost evaluations, and both approach the
    analytic exact gradient as the step shrinks."""
    g, aff, Y = small_problem(n=70, seed=4)
    st = oracle.Stage(1, *lam, 0.5)
    Z = oracle.exact_z(Y)
    grad, _ = oracle.exact_gradient(Y, aff.P_row, aff.P_col, aff.P_val64, st)
    for i, d in ((0, 0), (33, 1), (69, 0)):
        h = 1e-3
        Yp, Ym = Y.copy(), Y.copy()
        Yp[i, d] += h
        Ym[i, d] -= h
        full = (oracle.exact_cost(Yp, aff.P_row, aff.P_col, aff.P_val64, st)[0]
                - oracle.exact_cost(Ym, aff.P_row, aff.P_col, aff.P_val64, st)[0]) / (2 * h)
        step = oracle.exact_cost_central_difference(Y, aff.P_row, aff.P_col, aff.P_val64, st, i, d, h, Z)
        assert abs(step - full) <= 1e-8 * max(1.0, abs(full)), (i, d, step, full)
        small = oracle.exact_cost_central_difference(Y, aff.P_row, aff.P_col, aff.P_val64, st, i, d, 1e-6, Z)
        assert abs(small - grad[i, d]) <= 1e-7 * np.abs(grad).max(), (i, d, small, grad[i, d])


def test_interp_grad_pvals_central_differences():
    """dC/dp_e of the interpolated cost against central differences of
    interp_cost in each stored entry (Z from the grid does not depend on P)."""
    g, aff, Y = small_problem(n=60, seed=5)
    Y32 = Y.astype(np.float32)
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    gp = oracle.GridParams(min_boxes=8)
    dP = oracle.interp_grad_pvals(Y32, aff.P_row, aff.P_col, aff.P_val64, st, gp)
    order = np.argsort(-aff.P_val64)
    order = order[aff.P_val64[order] > 1e-12]  # entries that underflowed to 0 have no finite derivative
    for e in (order[0], order[len(order) // 2], order[-1]):
        h = aff.P_val64[e] * 1e-4
        Pp, Pm = aff.P_val64.copy(), aff.P_val64.copy()
        Pp[e] += h
        Pm[e] -= h
        fd = (oracle.interp_cost(Y32, aff.P_row, aff.P_col, Pp, st, gp)["total"]
              - oracle.interp_cost(Y32, aff.P_row, aff.P_col, Pm, st, gp)["total"]) / (2 * h)
        assert abs(fd - dP[e]) <= 1e-6 * abs(dP[e]), (e, fd, dP[e])
