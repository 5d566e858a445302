"""The grid convolution as split-BF16 DFT matrix products on the tensor cores
(conv_mode = LTSNET_CONV_DFT_GEMM), through the C ABI, against the FP64
oracle of the same interpolation (Sec. 2.3, Sec. 3.3): every term of the
gradient (repulsion R, entropy E, Z) within 1e-5 relative L2, the assembled
gradient within 1e-5 of the sum of its terms' norms, and the cost's Z and
entropy double sum likewise."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def grid32(ltlib):
    g = synth.grid2d(32, 32)
    aff = ltlib.affinities(g.row_ptr, g.col, 30.0)
    P = aff["P"]
    return g, P, tuple(t.cpu().numpy() for t in P)


def _layout_run(Pn, n, iters, seed=1):
    """Layouts along the oracle's own default run (iterations in `iters`)."""
    stages = oracle.default_stages(1000)
    sched = []
    for st in stages:
        sched += [st] * st.iters
    Y = synth.initial_layout(n, seed).astype(np.float64)
    upd = np.zeros_like(Y)
    gains = np.ones_like(Y)
    lr = oracle.auto_learning_rate(n)
    out = {}
    for it in range(max(iters) + 1):
        Y32 = Y.astype(np.float32)
        if it in iters:
            out[it] = Y32.copy()
        gr, _ = oracle.interp_gradient(Y32, Pn[0], Pn[1], Pn[2].astype(np.float64), sched[it], oracle.GridParams())
        Y, upd, gains = oracle.update(Y32.astype(np.float64), upd, gains, gr, sched[it].momentum, lr)
    return out


@pytest.fixture(scope="module")
def snaps(grid32):
    g, P, Pn = grid32
    return _layout_run(Pn, g.n, (0, 60, 300))


def _errors(lt, P, Pn, Y32, stage, params, gp):
    import torch

    grad, parts, terms = lt.gradient(P, torch.from_numpy(Y32).cuda(), stage, params, parts=True)
    ost = oracle.Stage(stage.iters, stage.lambda_kl, stage.lambda_c, stage.lambda_r, stage.exaggeration,
                       stage.momentum)
    gref, pr = oracle.interp_gradient(Y32, Pn[0], Pn[1], Pn[2].astype(np.float64), ost, gp)
    grad, parts, terms = grad.cpu().numpy(), parts.cpu().numpy(), terms.cpu().numpy()
    assert int(terms[2]) == pr["grid"].I
    n = Y32.shape[0]
    scale = (np.linalg.norm(4 * ost.lambda_kl * ost.exaggeration * pr["A"])
             + np.linalg.norm(4 * ost.lambda_kl * pr["S"] / pr["Z"] * pr["R"])
             + np.linalg.norm(ost.lambda_c / n * Y32.astype(np.float64))
             + np.linalg.norm(ost.lambda_r / n ** 2 * pr["E"]))
    return dict(grad=float(np.linalg.norm(grad - gref) / scale), R=rel(parts[:, 2:4], pr["R"]),
                E=rel(parts[:, 4:6], pr["E"]), Z=abs(terms[0] - pr["Z"]) / pr["Z"])


@pytest.mark.parametrize("which", [0, 60, 300])
def test_dft_gemm_gradient_grid32(ltlib, grid32, snaps, which):
    """Layouts of a default run on the 32x32 grid: the tiny start (grid of 50
    boxes over 1e-4), the spreading layout and a converged one."""
    g, P, Pn = grid32
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    errs = _errors(ltlib, P, Pn, snaps[which], st, ltlib.Params(conv_mode=1), oracle.GridParams())
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


@pytest.mark.parametrize("P_nodes,bw,minb,maxb", [(2, 0.25, 50, 640), (3, 0.1, 50, 640), (4, 0.25, 17, 500),
                                                  (5, 0.5, 50, 400), (3, 0.25, 50, 64)])
def test_dft_gemm_grid_settings(ltlib, grid32, snaps, P_nodes, bw, minb, maxb):
    """Other node counts, box widths and the box cap: grids from M = 100 to
    M = 648 nodes (the tile edges of every product fall at different places)."""
    g, P, Pn = grid32
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    params = ltlib.Params(nodes_per_box=P_nodes, box_width_max=bw, min_boxes=minb, max_boxes=maxb, conv_mode=1)
    gp = oracle.GridParams(nodes_per_box=P_nodes, box_width_max=bw, min_boxes=minb, max_boxes=maxb)
    errs = _errors(ltlib, P, Pn, snaps[300], st, params, gp)
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


def test_dft_gemm_equals_fft_form(ltlib, grid32, snaps):
    """The two convolution forms agree with each other as closely as each
    agrees with the oracle."""
    import torch

    g, P, Pn = grid32
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    Y = torch.from_numpy(snaps[300]).cuda()
    _, pa, ta = ltlib.gradient(P, Y, st, ltlib.Params(conv_mode=0), parts=True)
    _, pb, tb = ltlib.gradient(P, Y, st, ltlib.Params(conv_mode=1), parts=True)
    pa, pb = pa.cpu().numpy().astype(np.float64), pb.cpu().numpy().astype(np.float64)
    assert rel(pb[:, 2:4], pa[:, 2:4]) < 2 * TOL and rel(pb[:, 4:6], pa[:, 4:6]) < 2 * TOL
    assert abs(float(tb[0]) - float(ta[0])) < 2 * TOL * float(ta[0])


def test_dft_gemm_sbm_layout_large_grid(ltlib):
    """A 20,000-vertex SBM of the 100k recipe at a spread-out layout (extent
    about 60: 240 boxes, M = 720 nodes, FFT length 1440)."""
    import torch

    g = synth.sbm_powerlaw(20_000, 32, 12.0, 0.5, seed=2)
    aff = ltlib.affinities(g.row_ptr, g.col, 40.0)
    P = aff["P"]
    Pn = tuple(t.cpu().numpy() for t in P)
    Y32 = (np.random.default_rng(3).standard_normal((g.n, 2)) * 10).astype(np.float32)
    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    params = ltlib.Params(perplexity=40.0, conv_mode=1)
    errs = _errors(ltlib, P, Pn, Y32, st, params, oracle.GridParams(max_boxes=640))
    for key, v in errs.items():
        assert v < TOL, f"{key}: {v:.3e} ({errs})"


def test_dft_gemm_cost_terms(ltlib, grid32, snaps):
    """C_KL (through Z) and C_ENT (the entropy double sum by Parseval) from
    the tensor-core form against the oracle's interpolated cost."""
    g, P, Pn = grid32
    import torch

    st = ltlib.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    c, _ = ltlib.cost(P, torch.from_numpy(snaps[300]).cuda(), st, ltlib.Params(conv_mode=1))
    c = c.cpu().numpy()
    ref = oracle.interp_cost(snaps[300], Pn[0], Pn[1], Pn[2].astype(np.float64),
                             oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8), oracle.GridParams())
    assert abs(c[0] - ref["kl"]) <= TOL * abs(ref["kl"])
    assert abs(c[2] - ref["ent"]) <= TOL * abs(ref["ent"])


def test_dft_gemm_run_deterministic_and_final_cost(ltlib, grid32):
    """Whole runs with the tensor-core convolution: bit-identical from run to
    run, and the final layout's exact cost within 1% of the oracle run's."""
    import torch

    g, P, Pn = grid32
    Y0 = synth.initial_layout(g.n, 1)
    params = ltlib.Params(conv_mode=1)
    a, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), params)
    b, _ = ltlib.run(g.row_ptr, g.col, torch.from_numpy(Y0), params)
    assert torch.equal(a, b)
    Pv = Pn[2].astype(np.float64)
    Yo = oracle.run(Y0, Pn[0], Pn[1], Pv, oracle.default_stages(1000), oracle.GridParams())
    st = oracle.default_stages(1000)[-1]
    cg = oracle.exact_cost(a.cpu().numpy().astype(np.float64), Pn[0], Pn[1], Pv, st)[0]
    co = oracle.exact_cost(Yo.astype(np.float32).astype(np.float64), Pn[0], Pn[1], Pv, st)[0]
    assert abs(cg - co) <= 0.01 * abs(co), (cg, co)


def test_dft_gemm_rejected_with_plain_form(ltlib):
    import ctypes

    cp = ltlib.Params(conv_mode=1, plain=True).to_c()
    assert ltlib.lib().ltsnet_gradient_workspace_size(1000, ctypes.byref(cp)) == 0
    cp = ltlib.Params(conv_mode=2).to_c()
    assert ltlib.lib().ltsnet_gradient_workspace_size(1000, ctypes.byref(cp)) == 0
