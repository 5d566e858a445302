"""Parity of the GPU quadtree gradient (BH-tsNET Alg. 1, FIt-tsNET Alg. 2)
against the quadtree oracle, through the C ABI.

The GPU and the oracle build the same tree and open the same nodes (every
decision is taken in the same FP32 / fixed-point arithmetic), so the sums
differ only by FP32 accumulation: 1e-5 relative L2 per term, as for the
L-tsNET gradient, and the assembled gradient relative to the sum of its
terms' norms."""
import numpy as np
import pytest

import oracle
import synth
from oracle import quadtree

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    g = synth.grid2d(40, 35)
    ref = oracle.preprocess(g.row_ptr, g.col, 10.0)
    return g, ref


def layouts(n, seed):
    rng = np.random.default_rng(seed)
    yield "gauss", (rng.normal(size=(n, 2)) * 8).astype(np.float32)
    Y = (rng.normal(size=(n, 2)) * rng.choice([0.01, 1.0, 20.0], size=(n, 1))).astype(np.float32)
    Y[rng.integers(0, n, n // 20)] = Y[3]  # coincident points
    yield "clustered", Y


def gpu_P(lt, ref):
    import torch

    return (torch.from_numpy(ref.P_row).cuda(), torch.from_numpy(ref.P_col).cuda(),
            torch.from_numpy(ref.P_val64.astype(np.float32)).cuda())


ST_ARGS = (1, 1.0, 0.01, 0.6, 1.0, 0.8)
ST = oracle.Stage(*ST_ARGS)


@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_bh_matches_oracle(ltlib, case, theta):
    import torch

    g, ref = case
    P = gpu_P(ltlib, ref)
    pv = ref.P_val64.astype(np.float32).astype(np.float64)
    st = ltlib.Stage(*ST_ARGS)
    for name, Y in layouts(g.n, 3):
        grad, parts, (Z, S) = ltlib.gradient_quadtree(P, torch.from_numpy(Y).cuda(), st, theta=theta, variant="bh",
                                                      parts=True)
        go, d = quadtree.gradient(Y, ref.P_row, ref.P_col, pv, ST, theta, "bh")
        pt = parts.cpu().numpy()
        assert rel(pt[:, 0:2], d["A"]) < TOL, name
        assert rel(pt[:, 2:4], d["R"]) < TOL, name
        assert rel(pt[:, 4:6], d["E"]) < TOL, name
        assert Z == pytest.approx(d["Z"], rel=1e-6), name
        assert S == pytest.approx(d["S"], rel=1e-6), name
        scale = (np.linalg.norm(4 * d["A"]) + np.linalg.norm(4 * d["S"] / d["Z"] * d["R"])
                 + np.linalg.norm(0.6 / g.n ** 2 * d["E"]))
        assert np.linalg.norm(grad.cpu().numpy() - go) / scale < TOL, name


def test_bh_theta_zero_is_exact(ltlib, case):
    import torch

    g, ref = case
    P = gpu_P(ltlib, ref)
    Y = (np.random.default_rng(5).normal(size=(g.n, 2)) * 4).astype(np.float32)
    _, parts, (Z, _) = ltlib.gradient_quadtree(P, torch.from_numpy(Y).cuda(), ltlib.Stage(*ST_ARGS), theta=0.0,
                                               variant="bh", parts=True)
    empty = (np.zeros(g.n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    _, Rx, Ex, Zx = oracle.exact_sums(Y.astype(np.float64), *empty)
    pt = parts.cpu().numpy()
    assert rel(pt[:, 2:4], Rx) < TOL and rel(pt[:, 4:6], Ex) < TOL
    assert Z == pytest.approx(Zx, rel=1e-6)


def test_fit_matches_oracle(ltlib, case):
    import torch

    g, ref = case
    P = gpu_P(ltlib, ref)
    pv = ref.P_val64.astype(np.float32).astype(np.float64)
    st = ltlib.Stage(*ST_ARGS)
    for name, Y in layouts(g.n, 4):
        grad, parts, (Z, S) = ltlib.gradient_quadtree(P, torch.from_numpy(Y).cuda(), st, theta=0.5, variant="fit",
                                                      parts=True)
        _, gp = oracle.interp_gradient(Y, ref.P_row, ref.P_col, pv, ST, oracle.GridParams())
        go, d = quadtree.gradient(Y, ref.P_row, ref.P_col, pv, ST, 0.5, "fit", grid_parts=(gp["A"], gp["R"], gp["Z"]))
        pt = parts.cpu().numpy()
        assert rel(pt[:, 2:4], d["R"]) < TOL, name  # the grid's R
        assert rel(pt[:, 4:6], d["E"]) < TOL, name  # the quadtree's E
        assert Z == pytest.approx(gp["Z"], rel=1e-6), name
        scale = (np.linalg.norm(4 * d["A"]) + np.linalg.norm(4 * d["S"] / d["Z"] * d["R"])
                 + np.linalg.norm(0.6 / g.n ** 2 * d["E"]))
        assert np.linalg.norm(grad.cpu().numpy() - go) / scale < TOL, name


def test_bh_rgg1m_sampled_against_exact(ltlib):
    """The 1M-vertex RGG drawn by Pivot MDS (spread to unit scale): the
    quadtree sums at theta = 0.5 against the exact O(n) sums of 40 sampled
    points, within the approximation's error (a few percent)."""
    import torch

    g = synth.config_graph("rgg1m")
    Y, _, _ = ltlib.pivot_mds(g.row_ptr, g.col, 20, init_std=10.0)
    n = g.n
    P = (torch.from_numpy(np.arange(n + 1, dtype=np.int64)).cuda() * 0, torch.zeros(1, dtype=torch.int32).cuda(),
         torch.zeros(1, dtype=torch.float32).cuda())
    _, parts, (Z, _) = ltlib.gradient_quadtree(P, Y, ltlib.Stage(*ST_ARGS), theta=0.5, variant="bh", parts=True)
    pt = parts.cpu().numpy()
    Yh = Y.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(6)
    errs = []
    for i in rng.choice(n, 40, replace=False):
        d = Yh[i] - Yh
        d2 = (d * d).sum(1)
        d2[i] = np.inf
        q = 1.0 / (1.0 + d2)
        r = (q * q)[:, None] * d
        e = d / (quadtree.EPS_DEFAULT + d2)[:, None]
        errs.append(np.linalg.norm(pt[i, 2:4] - r.sum(0)) / np.linalg.norm(r.sum(0)))
        errs.append(np.linalg.norm(pt[i, 4:6] - e.sum(0)) / np.linalg.norm(e.sum(0)))
    assert np.median(errs) < 0.02 and np.max(errs) < 0.2
    assert np.isfinite(Z) and Z > 0


@pytest.mark.parametrize("variant", ["bh", "fit"])
def test_optimize_steps_match_oracle(ltlib, variant):
    """Eight descent steps of BH-tsNET / FIt-tsNET from the same spread-out
    start (entropy on): FP32 GPU against the FP64 oracle loop with the same
    gradient and step rule."""
    import torch

    g = synth.grid2d(24, 20)
    ref = oracle.preprocess(g.row_ptr, g.col, 10.0)
    P = gpu_P(ltlib, ref)
    pv = ref.P_val64.astype(np.float32).astype(np.float64)
    Y0 = (np.random.default_rng(8).normal(size=(g.n, 2)) * 3).astype(np.float32)
    params = ltlib.Params(perplexity=10.0, stages=[ltlib.Stage(8, 1.0, 0.01, 0.6, 1.0, 0.8)])
    Yg = torch.from_numpy(Y0.copy()).cuda()
    upd = torch.zeros_like(Yg)
    gains = torch.ones_like(Yg)
    ltlib.optimize_quadtree(P, Yg, upd, gains, 0, 8, params, theta=0.5, variant=variant)
    Y = Y0.astype(np.float64)
    u = np.zeros_like(Y)
    gn = np.ones_like(Y)
    lr = max(200.0, g.n / 12.0)
    st = oracle.Stage(8, 1.0, 0.01, 0.6, 1.0, 0.8)
    for _ in range(8):
        Y32 = Y.astype(np.float32)
        gp = None
        if variant == "fit":
            _, d = oracle.interp_gradient(Y32, ref.P_row, ref.P_col, pv, st, oracle.GridParams())
            gp = (d["A"], d["R"], d["Z"])
        grad, _ = quadtree.gradient(Y32, ref.P_row, ref.P_col, pv, st, 0.5, variant, grid_parts=gp)
        Y, u, gn = oracle.update(Y, u, gn, grad, 0.8, lr)
    assert rel(Yg.cpu().numpy(), Y) < 1e-4


def test_degenerate_drawings(ltlib):
    """All points at one position (zero extent: the domain side falls back
    to 1, every point in one depth-16 cell, every pair exact: q = 1 and zero
    forces), and two points."""
    import torch

    n = 50
    Y = np.full((n, 2), 3.25, np.float32)
    P = (torch.zeros(n + 1, dtype=torch.int64).cuda(), torch.zeros(1, dtype=torch.int32).cuda(),
         torch.zeros(1, dtype=torch.float32).cuda())
    _, parts, (Z, _) = ltlib.gradient_quadtree(P, torch.from_numpy(Y).cuda(), ltlib.Stage(*ST_ARGS), theta=0.5,
                                               variant="bh", parts=True)
    assert Z == n * (n - 1)
    assert np.all(parts.cpu().numpy()[:, 2:] == 0)
    Zp, R, E = quadtree.sums(Y, 0.5)
    assert Zp.sum() == Z
    Y2 = np.array([[0, 0], [1, 0]], np.float32)
    P2 = (torch.zeros(3, dtype=torch.int64).cuda(), torch.zeros(1, dtype=torch.int32).cuda(),
          torch.zeros(1, dtype=torch.float32).cuda())
    _, parts, (Z, _) = ltlib.gradient_quadtree(P2, torch.from_numpy(Y2).cuda(), ltlib.Stage(*ST_ARGS), theta=10.0,
                                               variant="bh", parts=True)
    assert Z == pytest.approx(1.0, rel=1e-7)
    assert np.allclose(parts.cpu().numpy()[:, 2:4], [[-0.25, 0], [0.25, 0]], rtol=1e-6)
