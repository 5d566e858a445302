"""The GPU evaluates the interpolated repulsion, entropy and Z sums in a
node-local arrangement (charges measured from each node, odd kernels K*dx,
Z by Parseval) instead of the FIt-SNE arrangement the oracle writes out
(charges 1, x, y, x^2+y^2 in absolute coordinates).  The two are the same
sums regrouped exactly; this test restates the node-local arrangement in FP64
numpy and checks it against the oracle to rounding, on layouts whose extent
spans five orders of magnitude."""
import numpy as np
import pytest

import oracle
import synth


def lagrange(u, P):
    w = np.ones((u.shape[0], P))
    for a in range(P):
        for b in range(P):
            if b != a:
                w[:, a] *= (u - (b + 0.5)) / (a - b)
    return w


def node_local_sums(Y32, gp):
    gi = oracle.grid_rule(Y32, gp)
    P, M, s = gp.nodes_per_box, gi.M, gi.s
    L = 2 * M
    n = Y32.shape[0]
    lo, h = np.float32(gi.lo), np.float32(gi.h)
    Y = Y32.astype(np.float64)
    bx = np.clip(np.floor((Y32[:, 0] - lo) / h).astype(int), 0, gi.I - 1)
    by = np.clip(np.floor((Y32[:, 1] - lo) / h).astype(int), 0, gi.I - 1)
    ux = (Y[:, 0] - gi.lo) / s - P * bx
    uy = (Y[:, 1] - gi.lo) / s - P * by
    wx, wy = lagrange(ux, P), lagrange(uy, P)
    S = np.zeros((4, L, L))
    for b in range(P):
        for a in range(P):
            w = wx[:, a] * wy[:, b]
            ex, ey = ux - (a + 0.5), uy - (b + 0.5)
            for c, q in enumerate([np.ones(n), ex, ey, ex * ex + ey * ey]):
                np.add.at(S[c], (P * by + b, P * bx + a), w * q)
    d = np.arange(L)
    ok = (d < M) | (d > L - M)
    d = np.where(d < M, d, d - L).astype(float)
    DX, DY = np.meshgrid(d, d)
    V = np.outer(ok, ok)
    d2 = s * s * (DX ** 2 + DY ** 2)
    K1 = np.where(V, 1 / (1 + d2), 0)
    K2 = K1 * K1
    Ke = np.where(V, 1 / (gp.eps + d2), 0)
    F = np.fft.fft2
    Sh = [F(S[c]) for c in range(4)]
    k1, k2, ke, k2x, k2y, kex, key = (F(K1), F(K2), F(Ke), F(K2 * DX), F(K2 * DY), F(Ke * DX), F(Ke * DY))

    def inv(a):
        return np.real(np.fft.ifft2(a))[:M, :M]

    F0, Fe0 = inv(k2 * Sh[0]), inv(ke * Sh[0])
    Vx, Vy = inv(k2x * Sh[0] - k2 * Sh[1]), inv(k2y * Sh[0] - k2 * Sh[2])
    Vex, Vey = inv(kex * Sh[0] - ke * Sh[1]), inv(key * Sh[0] - ke * Sh[2])
    zn = np.real(np.sum(np.conj(Sh[0]) * k1 * Sh[0] + 2 * s * s * (
        np.conj(Sh[1]) * (2 * k2x * Sh[0] - k2 * Sh[1]) + np.conj(Sh[2]) * (2 * k2y * Sh[0] - k2 * Sh[2])
        + np.conj(Sh[3]) * k2 * Sh[0]))) / (L * L)
    R = np.zeros((n, 2))
    E = np.zeros((n, 2))
    for b in range(P):
        for a in range(P):
            w = wx[:, a] * wy[:, b]
            ex, ey = ux - (a + 0.5), uy - (b + 0.5)
            t = (P * by + b, P * bx + a)
            R[:, 0] += w * (ex * F0[t] + Vx[t])
            R[:, 1] += w * (ey * F0[t] + Vy[t])
            E[:, 0] += w * (ex * Fe0[t] + Vex[t])
            E[:, 1] += w * (ey * Fe0[t] + Vey[t])
    return s * R, s * E, zn - n


@pytest.mark.parametrize("scale", [1e-4, 0.5, 3.0, 12.0])
@pytest.mark.parametrize("P", [2, 3, 5])
def test_node_local_form_equals_oracle(scale, P):
    g = synth.grid2d(12, 10)
    aff = oracle.preprocess(g.row_ptr, g.col, 5.0)
    Y = (np.random.default_rng(int(scale * 10) + P).standard_normal((g.n, 2)) * scale).astype(np.float32)
    gp = oracle.GridParams(nodes_per_box=P, min_boxes=12, max_boxes=60)
    st = oracle.Stage(1, 1.0, 0.01, 0.6, 1.0, 0.8)
    _, pr = oracle.interp_gradient(Y, aff.P_row, aff.P_col, aff.P_val64, st, gp)
    R, E, Z = node_local_sums(Y, gp)
    assert np.linalg.norm(R - pr["R"]) <= 1e-11 * np.linalg.norm(pr["R"])
    assert np.linalg.norm(E - pr["E"]) <= 1e-11 * np.linalg.norm(pr["E"])
    assert abs(Z - pr["Z"]) <= 1e-10 * abs(pr["Z"])
