"""GPU parity of the per-iteration gradient and of the descent loop against
the FP64 oracle with the same interpolation, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 GPU gradient vs FP64 oracle of the same interpolation, rel. L2
# Each term (attraction A, repulsion R, entropy E, Z) is compared on its own.
# The assembled gradient is compared relative to the sum of its terms' norms:
# near a stationary layout the gradient is a small difference of large terms
# and its own norm is no scale for FP32 rounding.


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def grid32(ltlib):
    g = synth.grid2d(32, 32)
    aff = ltlib.affinities(g.row_ptr, g.col, 30.0)
    P = aff["P"]
    Pn = tuple(t.cpu().numpy() for t in P)
    return g, P, Pn


@pytest.fixture(scope="module")
def snapshots(grid32):
    """Layouts along an oracle run on the 32x32 grid (iterations 0, 60, 300)."""
    g, P, Pn = grid32
    stages = oracle.default_stages(1000)
    Y = synth.initial_layout(g.n, 1).astype(np.float64)
    upd = np.zeros_like(Y)
    gains = np.ones_like(Y)
    lr = oracle.auto_learning_rate(g.n)
    out = {}
    sched = []
    for st in stages:
        sched += [st] * st.iters
    for it in range(301):
        Y32 = Y.astype(np.float32)
        if it in (0, 60, 300):
            out[it] = Y32.copy()
        gr, _ = oracle.interp_gradient(Y32, Pn[0], Pn[1], Pn[2].astype(np.float64), sched[it], oracle.GridParams())
        Y, upd, gains = oracle.update(Y32.astype(np.float64), upd, gains, gr, sched[it].momentum, lr)
    return out


def _compare(lt, P, Pn, Y32, stage, params, gp, plain=False):
    import torch

    params.plain = plain
    grad, parts, terms = lt.gradient(P, torch.from_numpy(Y32).cuda(), stage, params, parts=True)
    ost = oracle.Stage(stage.iters, stage.lambda_kl, stage.lambda_c, stage.lambda_r, stage.exaggeration,
                       stage.momentum)
    gref, pr = oracle.interp_gradient(Y32, Pn[0], Pn[1], Pn[2].astype(np.float64), ost, gp)
    grad = grad.cpu().numpy()
    parts = parts.cpu().numpy()
    terms = terms.cpu().numpy()
    gi = pr["grid"]
    assert int(terms[2]) == gi.I and float(terms[3]) == np.float32(gi.h)
    n = Y32.shape[0]
    scale = (np.linalg.norm(4 * ost.lambda_kl * ost.exaggeration * pr["A"])
             + np.linalg.norm(4 * ost.lambda_kl * pr["S"] / pr["Z"] * pr["R"])
             + np.linalg.norm(ost.lambda_c / n * Y32.astype(np.float64))
             + np.linalg.norm(ost.lambda_r / n ** 2 * pr["E"]))
    errs = dict(grad=float(np.linalg.norm(grad - gref) / scale), A=rel(parts[:, 0:2], pr["A"]),
                R=rel(parts[:, 2:4], pr["R"]), E=rel(parts[:, 4:6], pr["E"]), Z=abs(terms[0] - pr["Z"]) / pr["Z"])
    return errs


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("which", ["init", "spread", 60, 300])
def test_gradient_grid32(ltlib, grid32, snapshots, which, plain):
    g, P, Pn = grid32
    if which == "init":
        Y = synth.initial_layout(g.n, 1)
    elif which == "spread":
        Y = (np.random.default_rng(0).standard_normal((g.n, 2)) * 10).astype(np.float32)
    else:
        Y = snapshots[which]
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    errs = _compare(ltlib, P, Pn, Y, st, ltlib.Params(), oracle.GridParams(), plain)
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


@pytest.mark.parametrize("P_nodes,bw,minb,maxb", [(2, 1.0, 20, 640), (4, 0.5, 10, 500), (5, 2.0, 7, 400),
                                                  (3, 0.25, 3, 640)])
def test_gradient_grid_settings(ltlib, grid32, P_nodes, bw, minb, maxb):
    g, P, Pn = grid32
    Y = (np.random.default_rng(3).standard_normal((g.n, 2)) * 4).astype(np.float32)
    st = ltlib.Stage(1, 0.7, 0.3, 0.9, 4.0, 0.5)
    params = ltlib.Params(nodes_per_box=P_nodes, box_width_max=bw, min_boxes=minb, max_boxes=maxb)
    gp = oracle.GridParams(nodes_per_box=P_nodes, box_width_max=bw, min_boxes=minb, max_boxes=maxb)
    errs = _compare(ltlib, P, Pn, Y, st, params, gp)
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


def test_gradient_max_boxes_cap(ltlib, grid32):
    """An extent far above max_boxes * box_width_max: the cap widens the boxes."""
    g, P, Pn = grid32
    Y = (np.random.default_rng(5).standard_normal((g.n, 2)) * 40).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    params = ltlib.Params(max_boxes=96)
    gp = oracle.GridParams(max_boxes=96)
    errs = _compare(ltlib, P, Pn, Y, st, params, gp)
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


def test_gradient_sbm20k(ltlib):
    """n = 20,000 (several spread tiles and FFT lengths, ragged tail rows)."""
    g = synth.sbm([8000, 6000, 3000, 2000, 1001], 12.0, 5000, seed=3)
    aff = ltlib.affinities(g.row_ptr, g.col, 40.0)
    P = aff["P"]
    Pn = tuple(t.cpu().numpy() for t in P)
    Y = (np.random.default_rng(1).standard_normal((g.n, 2)) * 15).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    errs = _compare(ltlib, P, Pn, Y, st, ltlib.Params(perplexity=40.0), oracle.GridParams())
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


@pytest.mark.parametrize("P_nodes", [3, 5])
def test_gradient_crowded_boxes(ltlib, P_nodes):
    """Few boxes holding hundreds to thousands of points each (the summed-by-
    warps boxes, several segments per box), n = 20,000."""
    g = synth.sbm([8000, 6000, 3000, 2000, 1001], 12.0, 5000, seed=3)
    aff = ltlib.affinities(g.row_ptr, g.col, 30.0)
    P = aff["P"]
    Pn = tuple(t.cpu().numpy() for t in P)
    Y = (np.random.default_rng(7).standard_normal((g.n, 2)) * 3).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    params = ltlib.Params(nodes_per_box=P_nodes, box_width_max=100.0, min_boxes=8, max_boxes=400)
    gp = oracle.GridParams(nodes_per_box=P_nodes, box_width_max=100.0, min_boxes=8, max_boxes=400)
    errs = _compare(ltlib, P, Pn, Y, st, params, gp)
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


def test_gradient_reports_bad_column(ltlib):
    """A column index out of range in a caller-supplied P is reported as
    LTSNET_ERR_BAD_GRAPH (the gather itself stays in range)."""
    import torch

    n = 4
    P_row = torch.tensor([0, 1, 2, 3, 4], dtype=torch.int64).cuda()
    P_col = torch.tensor([1, 0, 3, 7], dtype=torch.int32).cuda()
    P_val = torch.full((4,), 0.25, dtype=torch.float32).cuda()
    Y = torch.tensor([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]], dtype=torch.float32).cuda()
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    with pytest.raises(ltlib.LtsnetError) as ei:
        ltlib.gradient((P_row, P_col, P_val), Y, st, ltlib.Params())
    assert ei.value.code == ltlib.ERR_BAD_GRAPH


def test_gradient_tiny(ltlib):
    """n = 2 and n = 3 (closed-form sized inputs), isolated vertex rows."""
    import torch

    for n in (2, 3, 5):
        Y = np.array([[0.3, -0.2], [-0.5, 0.4], [1.0, 1.0], [2.0, -1.0], [-1.5, 0.0]][:n], np.float32)
        P_row = np.array([0, 1, 2] + [2] * (n - 2), np.int64)[: n + 1]
        P_col = np.array([1, 0], np.int32)
        P_val = np.array([0.5, 0.5], np.float32)
        P = (torch.from_numpy(P_row).cuda(), torch.from_numpy(P_col).cuda(), torch.from_numpy(P_val).cuda())
        st = ltlib.Stage(1, 1.0, 0.5, 0.6, 1.0, 0.8)
        errs = _compare(ltlib, P, (P_row, P_col, P_val), Y, st, ltlib.Params(), oracle.GridParams())
        for key, v in errs.items():
            assert v < TOL, f"n={n} {key}: {v:.3e} ({errs})"


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_nonfinite_layout_is_reported(ltlib, grid32, bad):
    """A layout with one non-finite coordinate: ltsnet_gradient and
    ltsnet_optimize return LTSNET_ERR_NONFINITE through the workspace status
    word (every grid decision is clamped, so the bad point only poisons the
    sums), and the library stays usable for the next call."""
    import torch

    g, P, Pn = grid32
    Y = synth.initial_layout(g.n, 1) * 1e4
    Y[17, 1] = bad
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    with pytest.raises(ltlib.LtsnetError) as ei:
        ltlib.gradient(P, torch.from_numpy(Y).cuda(), st, ltlib.Params())
    assert ei.value.code == ltlib.ERR_NONFINITE
    Yd = torch.from_numpy(Y).cuda()
    with pytest.raises(ltlib.LtsnetError) as ei:
        ltlib.optimize(P, Yd, torch.zeros_like(Yd), torch.ones_like(Yd), 0, 5,
                       ltlib.Params(stages=ltlib.default_stages(5)))
    assert ei.value.code == ltlib.ERR_NONFINITE
    ok = synth.initial_layout(g.n, 1) * 1e4
    grad, _, _ = ltlib.gradient(P, torch.from_numpy(ok).cuda(), st, ltlib.Params())
    assert torch.isfinite(grad).all()


def _run_steps(lt, P, Y0, start, count, params, state=None):
    import torch

    Y = torch.from_numpy(Y0).cuda().clone() if state is None else state[0]
    upd = torch.zeros_like(Y) if state is None else state[1]
    gains = torch.ones_like(Y) if state is None else state[2]
    lt.optimize(P, Y, upd, gains, start, count, params)
    return Y, upd, gains


def test_optimize_deterministic_and_resumable(ltlib, grid32):
    g, P, Pn = grid32
    Y0 = synth.initial_layout(g.n, 1)
    params = ltlib.Params(stages=ltlib.default_stages(400))
    a = _run_steps(ltlib, P, Y0, 0, 400, params)
    b = _run_steps(ltlib, P, Y0, 0, 400, params)
    assert all(np.array_equal(x.cpu().numpy(), y.cpu().numpy()) for x, y in zip(a, b))
    c = _run_steps(ltlib, P, Y0, 0, 137, params)
    c = _run_steps(ltlib, P, Y0, 137, 263, params, state=c)
    assert all(np.array_equal(x.cpu().numpy(), y.cpu().numpy()) for x, y in zip(a, c))


def test_optimize_first_steps_match_oracle(ltlib, grid32):
    """Ten descent steps from the same start: FP32 GPU vs FP64 oracle."""
    g, P, Pn = grid32
    Y0 = synth.initial_layout(g.n, 2)
    params = ltlib.Params(stages=ltlib.default_stages(1000))
    Yg = _run_steps(ltlib, P, Y0, 0, 10, params)[0].cpu().numpy()
    Yo = oracle.run(Y0, Pn[0], Pn[1], Pn[2].astype(np.float64), oracle.default_stages(1000), oracle.GridParams(),
                    iters=10)
    assert rel(Yg, Yo) < 1e-4


def test_full_run_final_cost_grid32(ltlib, grid32):
    """Whole method on the 32x32 grid (u = 30, 1000 iterations): the final
    costs (exact FP64 cost of each final layout) agree within 1%."""
    import torch

    g, P, Pn = grid32
    Y0 = synth.initial_layout(g.n, 1)
    params = ltlib.Params(stages=ltlib.default_stages(1000))
    Yg, rc = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), params)
    Yg = Yg.cpu().numpy()
    Pv = Pn[2].astype(np.float64)
    Yo = oracle.run(Y0, Pn[0], Pn[1], Pv, oracle.default_stages(1000), oracle.GridParams())
    st = oracle.default_stages(1000)[-1]
    cg, _ = oracle.exact_cost(Yg.astype(np.float64), Pn[0], Pn[1], Pv, st)
    co, _ = oracle.exact_cost(Yo, Pn[0], Pn[1], Pv, st)
    assert abs(cg - co) / abs(co) < 0.01, (cg, co)


def test_run_host_matches_device(ltlib, grid32):
    import torch

    g, P, Pn = grid32
    Y0 = synth.initial_layout(g.n, 4)
    params = ltlib.Params(stages=ltlib.default_stages(120))
    Yd, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), params)
    Yh = Y0.copy()
    ltlib.run_host(g.row_ptr, g.col, Yh, params)
    assert np.array_equal(Yd.cpu().numpy(), Yh)


def _scipy_order(g):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order

    A = csr_matrix((np.ones(g.col.shape[0]), g.col, g.row_ptr), shape=(g.n, g.n))
    seen = np.zeros(g.n, bool)
    out = []
    for s in range(g.n):
        if seen[s]:
            continue
        o = breadth_first_order(A, s, directed=True, return_predecessors=False)
        seen[o] = True
        out.append(o)
    return np.concatenate(out)


@pytest.mark.parametrize("gname", ["grid", "islands", "tree", "rgg"])
def test_bfs_order_is_fifo_discovery_order(ltlib, gname):
    """The renumbering is the discovery order of a FIFO BFS (scipy's
    breadth_first_order), restarted at the smallest unvisited vertex."""
    g = {"grid": synth.grid2d(40, 25),
         "islands": synth.csr_from_edges(60, np.array([5, 6, 7, 30, 31, 40]), np.array([6, 7, 8, 31, 32, 41])),
         "tree": synth.random_recursive_tree(5000, 3), "rgg": synth.rgg(20000, seed=7, lcc=False)}[gname]
    order, inv, reordered = ltlib.bfs_order(g.row_ptr, g.col)
    assert reordered
    order = order.cpu().numpy()
    inv = inv.cpu().numpy()
    assert np.array_equal(order, _scipy_order(g))
    assert np.array_equal(inv[order], np.arange(g.n))


def test_run_with_and_without_reordering(ltlib, grid32):
    """Renumbering changes only the floating-point summation order: the final
    costs of the two runs agree within 1%."""
    import torch

    g, P, Pn = grid32
    Y0 = synth.initial_layout(g.n, 5)
    a, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), ltlib.Params(stages=ltlib.default_stages(600)))
    b, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0),
                     ltlib.Params(stages=ltlib.default_stages(600), reorder=False))
    st = oracle.default_stages(600)[-1]
    Pv = Pn[2].astype(np.float64)
    ca, _ = oracle.exact_cost(a.cpu().numpy().astype(np.float64), Pn[0], Pn[1], Pv, st)
    cb, _ = oracle.exact_cost(b.cpu().numpy().astype(np.float64), Pn[0], Pn[1], Pv, st)
    assert abs(ca - cb) / abs(cb) < 0.01, (ca, cb)


def test_run_compact_columns_match_int32_columns(ltlib, grid32):
    """ltsnet_run streams P in its packed layout (int16 column offsets, rows
    padded to multiples of 4 and interleaved within 32-entry blocks) when
    the offsets fit; one iteration must then agree with ltsnet_optimize on
    the same P in CSR form with int32 columns up to FP32 summation order (the
    lanes sum the entries of a row in different groups)."""
    import torch

    g, P, Pn = grid32
    Y0 = synth.initial_layout(g.n, 9) * 1e4  # spread out: every term matters
    params = ltlib.Params(stages=ltlib.default_stages(1), reorder=False)
    a, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), params)
    Y = torch.from_numpy(Y0).cuda().clone()
    upd = torch.zeros_like(Y)
    gains = torch.ones_like(Y)
    ltlib.optimize(P, Y, upd, gains, 0, 1, params)
    step = (Y - torch.from_numpy(Y0).cuda()).abs().max().item()
    assert step > 0
    assert (a - Y).abs().max().item() <= 1e-5 * step + 1e-6 * Y.abs().max().item()


@pytest.mark.parametrize("which", ["init", 300])
def test_cost_terms_match_oracle(ltlib, grid32, snapshots, which):
    """C_KL, C_CMP and C_ENT of ltsnet_cost against the oracle's cost with the
    same interpolation (exact sparse sums, Z and the entropy double sum from
    the grid)."""
    import torch

    g, P, Pn = grid32
    Y = snapshots[0] if which == "init" else snapshots[300]
    if which == "init":
        Y = (np.random.default_rng(2).standard_normal((g.n, 2)) * 3).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    c, dP = ltlib.cost(P, torch.from_numpy(Y).cuda(), st, ltlib.Params(), grad_pvals=True)
    c = c.cpu().numpy()
    ost = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    ref = oracle.interp_cost(Y, Pn[0], Pn[1], Pn[2].astype(np.float64), ost, oracle.GridParams())
    for k, key in enumerate(("kl", "cmp", "ent", "total")):
        assert abs(c[k] - ref[key]) <= 1e-5 * abs(ref[key]) + 1e-9, (key, c[k], ref[key])
    # dC/dp_e with the same Z
    rows = np.repeat(np.arange(g.n), np.diff(Pn[0]))
    d2 = np.sum((Y[rows].astype(np.float64) - Y[Pn[1]]) ** 2, axis=1)
    want = 1.0 * (np.log(Pn[2].astype(np.float64)) + 1.0 + np.log1p(d2) + np.log(ref["Z"]))
    got = dP.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want)), np.max(np.abs(got - want))


def _autograd_checks(lt, P, Pn, Y32, st, params, gp, coords, recompute):
    """LTsNetCost at Y32 against the oracle: dC/dY against the oracle's
    interpolated gradient (rel. L2 over the sum of the term norms, TOL) and
    against central differences of the oracle's EXACT cost on ``coords``,
    held to a bound derived from the interpolation error itself:
        |FD - dC/dY| <= |g_interp - g_exact| (oracle, at that coordinate)
                        + max |dC/dY - g_interp| + 1e-7 max |g|
    (FD of the FP64 exact cost with a 1e-5 step is exact to far better than
    the last term).  dC/dP_val against the oracle's interpolated derivative
    (TOL, entries with p > 0) and against central differences of the
    forward in 5 entries."""
    import torch

    ost = oracle.Stage(st.iters, st.lambda_kl, st.lambda_c, st.lambda_r, st.exaggeration, st.momentum)
    pv = Pn[2].astype(np.float64)
    Y = torch.from_numpy(Y32).cuda()
    F = lt.ltsnet_cost_fn()
    Yv = Y.clone().requires_grad_(True)
    Pv = P[2].clone().requires_grad_(True)
    F.apply(Yv, Pv, P[0], P[1], st, params, recompute).backward()
    gY = Yv.grad.cpu().numpy().astype(np.float64)
    gP = Pv.grad.cpu().numpy().astype(np.float64)
    n = Y32.shape[0]
    gi, pr = oracle.interp_gradient(Y32, Pn[0], Pn[1], pv, ost, gp)
    scale = (np.linalg.norm(4 * ost.lambda_kl * pr["A"]) + np.linalg.norm(4 * ost.lambda_kl * pr["S"] / pr["Z"] * pr["R"])
             + np.linalg.norm(ost.lambda_c / n * Y32.astype(np.float64))
             + np.linalg.norm(ost.lambda_r / n ** 2 * pr["E"]))
    assert np.linalg.norm(gY - gi) / scale <= TOL
    dPo = oracle.interp_grad_pvals(Y32, Pn[0], Pn[1], pv, ost, gp)
    pos = pv > 0
    assert rel(gP[pos], dPo[pos]) <= TOL
    assert np.array_equal(np.isfinite(gP), pos)
    Yd = Y32.astype(np.float64)
    rows = np.array(sorted({i for i, _ in coords}), np.int32)
    A, R, E = oracle.exact_rows(Yd, Pn[0], Pn[1], pv, rows)
    Z = oracle.exact_z(Yd)
    ge = dict(zip(rows.tolist(), oracle.assemble(Yd[rows], A, R, E, Z, pr["S"], ost, n)))
    dgpu = float(np.abs(gY - gi).max())
    gmax = float(np.abs(gY).max())
    for i, d in coords:
        fd = oracle.exact_cost_central_difference(Yd, Pn[0], Pn[1], pv, ost, i, d, 1e-5, Z)
        bound = abs(gi[i, d] - ge[i][d]) + dgpu + 1e-7 * gmax
        assert abs(fd - gY[i, d]) <= bound, (i, d, fd, gY[i, d], bound)
    rng = np.random.default_rng(3)
    for e in rng.choice(np.nonzero(pv > 1e-10)[0], 5, replace=False):
        h = float(P[2][e]) * 1e-2
        Pp, Pm = P[2].clone(), P[2].clone()
        Pp[e] += h
        Pm[e] -= h
        cp = F.apply(Y, Pp, P[0], P[1], st, params).item()
        cm = F.apply(Y, Pm, P[0], P[1], st, params).item()
        fd = (cp - cm) / (Pp[e] - Pm[e]).item()
        assert abs(fd - gP[e]) <= 1e-3 * abs(gP[e]) + 1e-6, (e, fd, gP[e])


@pytest.mark.parametrize("recompute", [False, True])
def test_cost_autograd_grid32(ltlib, grid32, snapshots, recompute):
    """The autograd wrapper on the 32x32 grid at iteration 300 of a default
    run, with the default grid and with a finer one (where the interpolation
    error, and with it the finite-difference bound, is smaller)."""
    g, P, Pn = grid32
    Y32 = snapshots[300]
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    rng = np.random.default_rng(5)
    coords = [(int(i), int(d)) for i, d in zip(rng.choice(g.n, 16, replace=False), rng.integers(0, 2, 16))]
    for bw in (0.25, 0.1):
        params = ltlib.Params(box_width_max=bw)
        gp = oracle.GridParams(box_width_max=bw, max_boxes=640)
        _autograd_checks(ltlib, P, Pn, Y32, st, params, gp, coords, recompute)


def test_cost_autograd_rejects_exaggeration(ltlib, grid32, snapshots):
    import torch

    g, P, Pn = grid32
    F = ltlib.ltsnet_cost_fn()
    Y = torch.from_numpy(snapshots[60]).cuda().requires_grad_(True)
    with pytest.raises(ValueError):
        F.apply(Y, P[2], P[0], P[1], ltlib.Stage(1, 1.0, 0.01, 0.0, 12.0, 0.5), ltlib.Params())


@pytest.mark.parametrize("mode", [0, 1])
def test_run_batched_equals_single_runs(ltlib, mode):
    """ltsnet_run_batched over graphs of several kinds and sizes, with fewer
    workers than graphs -- the one-launch form (every phase one launch over
    all graphs, two launch shapes) and the per-graph form -- gives every
    graph exactly the layout ltsnet_run gives it alone; the one-launch form
    also reports each graph's largest box count, equal to its own run's.
    The star's centre has a row of P longer than the fused kernel's groups
    take, summed in chunks in both forms."""
    import torch

    star = synth.csr_from_edges(2501, np.zeros(2500, np.int64), np.arange(1, 2501, dtype=np.int64), "star2500")
    graphs = [synth.grid2d(20, 30), synth.random_recursive_tree(900, 5), synth.sbm([300, 250, 200], 9.5, 40, 7),
              synth.grid2d(9, 7), star, synth.rgg(1500, seed=9, lcc=True), synth.random_recursive_tree(150, 2)]
    Y0s = [synth.initial_layout(g.n, 11 + i) for i, g in enumerate(graphs)]
    params = ltlib.Params(stages=ltlib.default_stages(120))
    single = [ltlib.run(g.row_ptr, g.col, torch.from_numpy(y0), params)[0] for g, y0 in zip(graphs, Y0s)]
    shapes = [(0, 0), (1, 3)] if mode == 0 else [(0, 0)]
    for fb, sb in shapes:
        Y, off, boxes = ltlib.run_batched(graphs, Y0s, params, workers=3, mode=mode, fft_blocks=fb,
                                          spread_blocks=sb, return_boxes=True)
        for i in range(len(graphs)):
            assert torch.equal(Y[off[i]:off[i + 1]], single[i]), (mode, fb, sb, i)
        if mode == 0:
            assert np.all(boxes >= params.min_boxes) and np.all(boxes <= params.max_boxes)
        else:
            assert np.all(boxes == -1)


def test_run_batched_half_size_fft_blocks_equal_single_runs(ltlib):
    """With grid caps small enough for one column of the largest grid to fit
    in half of an SM's shared memory, the one-launch form runs its FFT passes
    as two 256-thread blocks per SM; every graph still gets exactly the
    layout ltsnet_run gives it alone (which uses one 512-thread block per SM),
    the long row of a star included."""
    import torch

    star = synth.csr_from_edges(2501, np.zeros(2500, np.int64), np.arange(1, 2501, dtype=np.int64), "star2500")
    graphs = [synth.grid2d(20, 30), synth.random_recursive_tree(900, 5), star, synth.sbm([300, 250, 200], 9.5, 40, 7)]
    Y0s = [synth.initial_layout(g.n, 31 + i) for i, g in enumerate(graphs)]
    params = ltlib.Params(stages=ltlib.default_stages(120), max_boxes=200)
    single = [ltlib.run(g.row_ptr, g.col, torch.from_numpy(y0), params)[0] for g, y0 in zip(graphs, Y0s)]
    for fb in (0, 3):
        Y, off = ltlib.run_batched(graphs, Y0s, params, workers=2, mode=0, fft_blocks=fb)
        for i in range(len(graphs)):
            assert torch.equal(Y[off[i]:off[i + 1]], single[i]), (fb, i)


def test_run_batched_per_graph_caps(ltlib):
    """Per-graph grid caps (ltsnet_batch_config.max_boxes): each graph of the
    batch runs exactly as ltsnet_run does with its own cap, in both forms,
    whether the cap binds (small caps) or not; an entry of 0 takes the
    parameters' cap; an out-of-range cap is rejected."""
    import torch

    graphs = [synth.grid2d(20, 30), synth.random_recursive_tree(900, 5), synth.sbm([300, 250, 200], 9.5, 40, 7),
              synth.grid2d(9, 7)]
    Y0s = [synth.initial_layout(g.n, 21 + i) for i, g in enumerate(graphs)]
    base = dict(stages=ltlib.default_stages(120), min_boxes=4, max_boxes=96)
    caps = [6, 0, 40, 9]
    single = []
    for g, y0, c in zip(graphs, Y0s, caps):
        q = ltlib.Params(**{**base, "max_boxes": c if c > 0 else base["max_boxes"]})
        single.append(ltlib.run(g.row_ptr, g.col, torch.from_numpy(y0), q)[0])
    params = ltlib.Params(**base)
    for mode in (0, 1):
        Y, off, boxes = ltlib.run_batched(graphs, Y0s, params, workers=2, mode=mode, return_boxes=True,
                                          max_boxes=caps)
        for i in range(len(graphs)):
            assert torch.equal(Y[off[i]:off[i + 1]], single[i]), (mode, i)
        if mode == 0:
            eff = np.where(np.array(caps) > 0, caps, base["max_boxes"])
            assert np.all(boxes <= eff)
            assert boxes[0] == 6 and boxes[3] == 9, boxes  # the small caps bind
    with pytest.raises(ltlib.LtsnetError):
        ltlib.run_batched(graphs, Y0s, params, workers=2, mode=0, max_boxes=[6, 0, 40, 100000])
    with pytest.raises(ltlib.LtsnetError):
        ltlib.run_batched(graphs, Y0s, params, workers=2, mode=0, max_boxes=[6, 0, 40, 2])  # below min_boxes


def test_run_batched_argument_checks(ltlib):
    graphs = [synth.grid2d(6, 6), synth.grid2d(5, 7)]
    Y0s = [synth.initial_layout(g.n, 1) for g in graphs]
    for params in (ltlib.Params(stages=ltlib.default_stages(10), plain=True),
                   ltlib.Params(stages=ltlib.default_stages(10), conv_mode=1)):
        with pytest.raises(ltlib.LtsnetError):
            ltlib.run_batched(graphs, Y0s, params, workers=2, mode=0)
    # both forms accept what a single run accepts
    ltlib.run_batched(graphs, Y0s, ltlib.Params(stages=ltlib.default_stages(10), plain=True), workers=2, mode=1)


def test_run_step_rgg1m_matches_oracle(ltlib):
    """The benchmark's workload at full size (RGG, n = 999,019) through
    ltsnet_run -- breadth-first renumbering, packed int16 P, the kernels the
    benchmark times -- for one iteration from a spread-out layout, against
    the oracle's interpolated gradient and update rule on the same P (the
    GPU's C0 in the original numbering, checked separately)."""
    import torch

    g = synth.config_graph("rgg1m")
    aff = ltlib.affinities(g.row_ptr, g.col, 30.0)
    Pn = tuple(t.cpu().numpy() for t in aff["P"])
    Y0 = (np.random.default_rng(12).standard_normal((g.n, 2)) * 12).astype(np.float32)
    params = ltlib.Params(perplexity=30.0, stages=[ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)])
    Y1, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), params)
    step = Y1.cpu().numpy().astype(np.float64) - Y0
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    gref, pr = oracle.interp_gradient(Y0, Pn[0], Pn[1], Pn[2].astype(np.float64), st, oracle.GridParams(max_boxes=640))
    lr = oracle.auto_learning_rate(g.n)
    Yr, _, _ = oracle.update(Y0.astype(np.float64), np.zeros_like(gref), np.ones_like(gref), gref, st.momentum, lr)
    sref = Yr - Y0
    n = g.n
    scale = (np.linalg.norm(4 * st.lambda_kl * st.exaggeration * pr["A"])
             + np.linalg.norm(4 * st.lambda_kl * pr["S"] / pr["Z"] * pr["R"])
             + np.linalg.norm(st.lambda_c / n * Y0.astype(np.float64))
             + np.linalg.norm(st.lambda_r / n ** 2 * pr["E"]))
    # the first step is -lr * 1.2 * g (gains start at 1 and grow by 0.2;
    # the previous update is 0)
    err = float(np.linalg.norm(step - sref) / (lr * 1.2 * scale))
    assert err < 1e-5, err


def _bfs_ball(g, root: int, size: int):
    return synth.bfs_ball(g, root, size)[0]


@pytest.fixture(scope="module")
def ba_ball():
    """The induced subgraph on a 50,000-vertex BFS ball, from a seeded root,
    of the Barabasi-Albert graph (n = 4e6, 4 edges per new vertex)."""
    g = synth.config_graph("ba4m")
    root = int(np.random.default_rng(21).integers(g.n))
    return _bfs_ball(g, root, 50_000)


def test_ba4m_ball_pipeline_matches_oracle(ltlib, ba_ball):
    """The cfg-5 graph's 50,000-vertex BFS ball, perplexity 50: C0 and the
    gradient on both sides (GPU through the ABI, the oracle on its own C0),
    hubs and all."""
    import torch

    sub = ba_ball
    aff = ltlib.affinities(sub.row_ptr, sub.col, 50.0)
    ref = oracle.preprocess(sub.row_ptr, sub.col, 50.0)
    P = aff["P"]
    Pn = tuple(t.cpu().numpy() for t in P)
    assert np.array_equal(Pn[0], ref.P_row) and np.array_equal(Pn[1], ref.P_col)
    np.testing.assert_allclose(Pn[2], ref.P_val64, rtol=1e-6, atol=0)
    Y = (np.random.default_rng(4).standard_normal((sub.n, 2)) * 10).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    errs = _compare(ltlib, P, (ref.P_row, ref.P_col, ref.P_val64), Y, st, ltlib.Params(perplexity=50.0),
                    oracle.GridParams())
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


def test_cost_autograd_sbm100k_64_coordinates(ltlib):
    """The autograd wrapper on the 100,000-vertex SBM (perplexity 40) at a
    spread-out layout: dC/dY against the oracle's interpolated gradient and
    against central differences of the oracle's exact cost on 64 random
    coordinates (bound from the interpolation error), dC/dP_val against the
    oracle and central differences; in the recompute mode."""
    g = synth.config_graph("sbm100k")
    aff = ltlib.affinities(g.row_ptr, g.col, 40.0)
    P = aff["P"]
    Pn = tuple(t.cpu().numpy() for t in P)
    rng = np.random.default_rng(64)
    Y32 = (rng.standard_normal((g.n, 2)) * 8).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    params = ltlib.Params(perplexity=40.0)
    gp = oracle.GridParams(max_boxes=params.max_boxes)
    coords = [(int(i), int(d)) for i, d in zip(rng.choice(g.n, 64, replace=False), rng.integers(0, 2, 64))]
    _autograd_checks(ltlib, P, Pn, Y32, st, params, gp, coords, recompute=True)


def test_run_step_ba_ball_long_rows_match_oracle(ltlib, ba_ball):
    """ltsnet_run on the cfg-5 ball for one iteration: the hubs' rows of P are
    longer than one 8-lane group takes (they are summed in chunks by whole
    warps); the step agrees with the oracle's gradient and update."""
    import torch

    sub = ba_ball
    aff = ltlib.affinities(sub.row_ptr, sub.col, 50.0)
    Pn = tuple(t.cpu().numpy() for t in aff["P"])
    assert np.diff(Pn[0]).max() > 2048  # long rows present
    Y0 = (np.random.default_rng(13).standard_normal((sub.n, 2)) * 8).astype(np.float32)
    params = ltlib.Params(perplexity=50.0, stages=[ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)])
    Y1, _ = ltlib.run(sub.row_ptr, sub.col, torch.from_numpy(Y0), params)
    step = Y1.cpu().numpy().astype(np.float64) - Y0
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    gref, pr = oracle.interp_gradient(Y0, Pn[0], Pn[1], Pn[2].astype(np.float64), st, oracle.GridParams(max_boxes=640))
    lr = oracle.auto_learning_rate(sub.n)
    Yr, _, _ = oracle.update(Y0.astype(np.float64), np.zeros_like(gref), np.ones_like(gref), gref, st.momentum, lr)
    n = sub.n
    scale = (np.linalg.norm(4 * st.lambda_kl * st.exaggeration * pr["A"])
             + np.linalg.norm(4 * st.lambda_kl * pr["S"] / pr["Z"] * pr["R"])
             + np.linalg.norm(st.lambda_c / n * Y0.astype(np.float64))
             + np.linalg.norm(st.lambda_r / n ** 2 * pr["E"]))
    err = float(np.linalg.norm(step - (Yr - Y0)) / (lr * 1.2 * scale))
    assert err < 1e-5, err


def test_run_step_far_columns_match_oracle(ltlib):
    """ltsnet_run on a graph whose columns of P lie further than the int16
    range from their rows even after the breadth-first renumbering (a star
    with 40,000 leaves: the centre and the leaves every leaf lists have rows
    of about 40,000 entries), so P is streamed in the packed layout with
    int32 columns and the long rows are summed in chunks; one step agrees
    with the oracle's gradient and update."""
    import torch

    leaves = 40_000
    g = synth.csr_from_edges(leaves + 1, np.zeros(leaves, np.int64), np.arange(1, leaves + 1, dtype=np.int64),
                             "star40000")
    aff = ltlib.affinities(g.row_ptr, g.col, 30.0)
    Pn = tuple(t.cpu().numpy() for t in aff["P"])
    _, inv, reordered = ltlib.bfs_order(g.row_ptr, g.col)
    invn = inv.cpu().numpy().astype(np.int64) if reordered else np.arange(g.n, dtype=np.int64)
    rows = np.repeat(np.arange(g.n), np.diff(Pn[0]))
    assert np.abs(invn[Pn[1].astype(np.int64)] - invn[rows]).max() > 32767  # int32 columns
    assert np.diff(Pn[0]).max() > 2048  # long rows present
    Y0 = (np.random.default_rng(17).standard_normal((g.n, 2)) * 8).astype(np.float32)
    params = ltlib.Params(perplexity=30.0, stages=[ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)])
    Y1, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), params)
    step = Y1.cpu().numpy().astype(np.float64) - Y0
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    gref, pr = oracle.interp_gradient(Y0, Pn[0], Pn[1], Pn[2].astype(np.float64), st, oracle.GridParams())
    lr = oracle.auto_learning_rate(g.n)
    Yr, _, _ = oracle.update(Y0.astype(np.float64), np.zeros_like(gref), np.ones_like(gref), gref, st.momentum, lr)
    n = g.n
    scale = (np.linalg.norm(4 * st.lambda_kl * st.exaggeration * pr["A"])
             + np.linalg.norm(4 * st.lambda_kl * pr["S"] / pr["Z"] * pr["R"])
             + np.linalg.norm(st.lambda_c / n * Y0.astype(np.float64))
             + np.linalg.norm(st.lambda_r / n ** 2 * pr["E"]))
    err = float(np.linalg.norm(step - (Yr - Y0)) / (lr * 1.2 * scale))
    assert err < 1e-5, err


def test_rgg1m_ball20k_parity_both_forms_and_exact(ltlib, capsys):
    """The benchmark graph's 20,000-vertex BFS ball (cfg 3's error on a
    20k-vertex subsample), at iteration 300 of the oracle's own run on it:
    every gradient term of both convolution forms against the oracle's
    interpolation (1e-5), and the oracle's interpolation against the exact
    O(n^2) sums (5e-3, the accuracy contract); the measured errors are
    printed."""
    import torch

    g = synth.config_graph("rgg1m")
    root = int(np.random.default_rng(31).integers(g.n))
    sub, _ = synth.bfs_ball(g, root, 20_000)
    aff = ltlib.affinities(sub.row_ptr, sub.col, 30.0)
    P = aff["P"]
    Pn = tuple(t.cpu().numpy() for t in P)
    ref = oracle.preprocess(sub.row_ptr, sub.col, 30.0)
    assert np.array_equal(Pn[0], ref.P_row) and np.array_equal(Pn[1], ref.P_col)
    pv = Pn[2].astype(np.float64)
    Y = oracle.run(synth.initial_layout(sub.n, 3), Pn[0], Pn[1], pv, oracle.default_stages(1000),
                   oracle.GridParams(), iters=300).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    out = {}
    for conv in (0, 1):
        errs = _compare(ltlib, P, Pn, Y, st, ltlib.Params(conv_mode=conv), oracle.GridParams())
        out[conv] = errs
        for key, v in errs.items():
            assert v < TOL, f"conv {conv} {key}: {v:.3e} ({errs})"
    ost = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    Yd = Y.astype(np.float64)
    A, R, E = oracle.exact_rows(Yd, Pn[0], Pn[1], pv, np.arange(sub.n, dtype=np.int32))
    Z = oracle.exact_z(Yd)
    _, pr = oracle.interp_gradient(Y, Pn[0], Pn[1], pv, ost, oracle.GridParams())
    acc = dict(R=rel(pr["R"], R), E=rel(pr["E"], E), Z=abs(pr["Z"] - Z) / Z)
    for key, v in acc.items():
        assert v <= 5e-3, (key, acc)
    with capsys.disabled():
        print(f"\nrgg1m ball20k (extent {float(Y.max() - Y.min()):.1f}): fft {out[0]}\n  dft_gemm {out[1]}\n"
              f"  interp vs exact {acc}")
