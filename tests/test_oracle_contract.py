"""The accuracy contract of the interpolation (Sec. 2.3 "four sums", Sec. 3.3
entropy sums, Alg. 3 loop), on the oracle alone: at the default grid settings
the interpolated sums stay within 5e-3 of the exact O(n^2) sums along a whole
run, and an interpolated run ends at the cost of an exact-gradient run.

Normalisation.  Each interpolated quantity -- the repulsion sums R, the
entropy sums E and Z -- is compared with its exact value relative to its own
exact norm.  The assembled gradient is compared relative to the sum of its
terms' norms (attraction, repulsion, compression, entropy), the scale the GPU
parity tests use as well.  Its own norm is no scale: near a stationary layout
the gradient is a small difference of large terms, and relative to its own
norm the error of any fixed grid grows without bound as the run converges (on
the 32x32 grid at iteration 999: 1.0 with 3 nodes and boxes of width 0.42,
still 1.4e-3 with 5 nodes and 100 boxes).
"""
import numpy as np
import pytest

import oracle
import synth

CONTRACT = 5e-3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _run(P_row, P_col, P_val, Y0, stages, gp, exact=False, keep=()):
    """The oracle's Alg. 3 loop (oracle.run), keeping the FP32 layouts at the
    iterations in ``keep``."""
    n = Y0.shape[0]
    lr = oracle.auto_learning_rate(n)
    Y = np.asarray(Y0, np.float64).copy()
    upd = np.zeros_like(Y)
    gains = np.ones_like(Y)
    sched = []
    for st in stages:
        sched += [st] * st.iters
    snaps = {}
    for it, st in enumerate(sched):
        Y32 = Y.astype(np.float32)
        if it in keep:
            snaps[it] = (Y32.copy(), st)
        if exact:
            g, _ = oracle.exact_gradient(Y32.astype(np.float64), P_row, P_col, P_val, st, gp.eps)
        else:
            g, _ = oracle.interp_gradient(Y32, P_row, P_col, P_val, st, gp)
        Y, upd, gains = oracle.update(Y32.astype(np.float64), upd, gains, g, st.momentum, lr)
    return Y, snaps


def _errors(Y32, P_row, P_col, P_val, st, gp, rows=None):
    """INTERP against EXACT at Y32 on the target rows ``rows`` (all rows if
    None): per-term relative errors and the gradient's error relative to the
    sum of the term norms."""
    n = Y32.shape[0]
    Y = Y32.astype(np.float64)
    rows = np.arange(n, dtype=np.int32) if rows is None else rows
    A, R, E = oracle.exact_rows(Y, P_row, P_col, P_val, rows, gp.eps)
    Z = oracle.exact_z(Y)
    S = float(np.sum(P_val))
    g_exact = oracle.assemble(Y[rows], A, R, E, Z, S, st, n)
    g, parts = oracle.interp_gradient(Y32, P_row, P_col, P_val, st, gp)
    scale = (np.linalg.norm(4 * st.lambda_kl * st.exaggeration * A) + np.linalg.norm(4 * st.lambda_kl * S / Z * R)
             + np.linalg.norm(st.lambda_c / n * Y[rows]) + np.linalg.norm(st.lambda_r / n ** 2 * E))
    return dict(R=rel(parts["R"][rows], R), E=rel(parts["E"][rows], E), Z=abs(parts["Z"] - Z) / Z,
                grad=float(np.linalg.norm(g[rows] - g_exact) / scale), own=rel(g[rows], g_exact),
                ext=float(Y32.max() - Y32.min()), I=parts["grid"].I)


@pytest.fixture(scope="module")
def grid32_run():
    g = synth.grid2d(32, 32)
    aff = oracle.preprocess(g.row_ptr, g.col, 30.0)
    Y0 = synth.initial_layout(g.n, 1)
    gp = oracle.GridParams()
    Y, snaps = _run(aff.P_row, aff.P_col, aff.P_val64, Y0, oracle.default_stages(1000), gp, keep=(0, 300, 600, 999))
    return aff, Y0, Y, snaps


def test_default_grid_settings_are_the_library_readings():
    gp = oracle.GridParams()
    assert (gp.nodes_per_box, gp.box_width_max, gp.min_boxes) == (3, 0.25, 50)


def test_interp_matches_exact_along_a_run_grid32(grid32_run):
    """32x32 grid (perplexity 30): layouts at iterations 0, 300, 600 and 999
    of a default run, every row."""
    aff, _, _, snaps = grid32_run
    gp = oracle.GridParams()
    for it, (Y32, st) in snaps.items():
        e = _errors(Y32, aff.P_row, aff.P_col, aff.P_val64, st, gp)
        for key in ("R", "E", "Z", "grad"):
            assert e[key] <= CONTRACT, (it, e)


def test_interp_run_ends_at_the_cost_of_an_exact_run_grid32(grid32_run):
    """The interpolated run and a run with the exact O(n^2) gradient from the
    same start: the exact cost of the two final layouts within 1%."""
    aff, Y0, Y_interp, _ = grid32_run
    gp = oracle.GridParams()
    Y_exact, _ = _run(aff.P_row, aff.P_col, aff.P_val64, Y0, oracle.default_stages(1000), gp, exact=True)
    st = oracle.default_stages(1000)[-1]
    c_interp = oracle.exact_cost(Y_interp.astype(np.float32).astype(np.float64), aff.P_row, aff.P_col,
                                 aff.P_val64, st)[0]
    c_exact = oracle.exact_cost(Y_exact.astype(np.float32).astype(np.float64), aff.P_row, aff.P_col,
                                aff.P_val64, st)[0]
    assert abs(c_interp - c_exact) <= 0.01 * abs(c_exact), (c_interp, c_exact)


@pytest.fixture(scope="module")
def sbm20k_run():
    """An SBM of the 100,000-vertex recipe scaled to 20,000 vertices (32
    power-law blocks, in-block degree 12, cross degree 0.5, perplexity 40),
    a default run, layouts at iterations 300 and 999."""
    g = synth.sbm_powerlaw(20_000, 32, 12.0, 0.5, seed=2)
    aff = oracle.preprocess(g.row_ptr, g.col, 40.0)
    Y0 = synth.initial_layout(g.n, 2)
    _, snaps = _run(aff.P_row, aff.P_col, aff.P_val64, Y0, oracle.default_stages(1000), oracle.GridParams(),
                    keep=(300, 999))
    return aff, snaps


def test_interp_matches_exact_along_a_run_sbm20k(sbm20k_run):
    """Every row of the clustered SBM layouts (tight blocks: the hardest case
    for the narrow entropy kernel)."""
    aff, snaps = sbm20k_run
    gp = oracle.GridParams()
    for it, (Y32, st) in snaps.items():
        e = _errors(Y32, aff.P_row, aff.P_col, aff.P_val64, st, gp)
        for key in ("R", "E", "Z", "grad"):
            assert e[key] <= CONTRACT, (it, e)


def test_boxes_twice_as_wide_break_the_contract(sbm20k_run):
    """The reason for the default box width: boxes up to 0.5 wide (54 boxes
    on the final SBM layout) leave the entropy sums 1.7e-2 off -- the
    entropy kernel is only sqrt(eps) = 0.22 wide -- while the repulsion,
    whose kernel is 1 wide, still passes."""
    aff, snaps = sbm20k_run
    Y32, st = snaps[999]
    e = _errors(Y32, aff.P_row, aff.P_col, aff.P_val64, st, oracle.GridParams(box_width_max=0.5))
    assert e["E"] > CONTRACT and e["R"] <= CONTRACT, e
