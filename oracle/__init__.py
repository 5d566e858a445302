"""FP64 CPU oracle for the L-tsNET gradient hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The GPU library never imports it
and it imports nothing from the GPU library; the only module the two sides
share is ``synth`` (seeded inputs, none of the method's arithmetic).

The heavy loops live in ``ltsnet_oracle.c`` (plain C, FP64, built into
``liboracle.so`` with -ffp-contract=off); this module marshals numpy arrays
into it and writes the few vector formulas (gradient assembly, update) out in
numpy.  The only library primitive used as a step is numpy's FFT, for the
grid convolution at grid sizes where the direct O(M^4) sum is too slow; the
two are cross-checked in the tests.

Paper: Meidiana, Hong, Ma, "BH-tsNET, FIt-tsNET, L-tsNET: Fast tsNET
Algorithms for Large Graph Drawing" (arXiv 2509.19785).  Section, equation and
algorithm citations below refer to it.

Parity status: every function here is pinned by a test in
``tests/test_oracle_*.py`` except the optimiser constants and the stage
schedule (``update`` and ``default_stages``), which the paper does not give
(Alg. 3 says only "move each vertex in the direction of dC/dv"): parity
unpinned for those; the GPU and the oracle take them as the same inputs.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ltsnet_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

EPS_DEFAULT = 1.0 / 20.0  # Sec. 3.3: eps = 1/20, as in tsNET


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        # OpenMP splits only loops over independent rows (each row summed by
        # one thread in a fixed order): results do not depend on the threads.
        # Without an OpenMP runtime the same source builds serial.
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp]
        try:
            subprocess.check_call(base + ["-fopenmp", _SRC, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + [_SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        L.or_partial_bfs.argtypes = [i32, P, P, i32, i32, i32, P, P, P]
        L.or_calibrate.argtypes = [i32, i32, P, P, f64, f64, i32, P, P, P]
        L.or_symmetrize.argtypes = [i32, i32, P, P, P, P, P, P, i64]
        L.or_symmetrize.restype = i64
        L.or_exact_sums.argtypes = [i32, P, P, P, P, f64, P, P, P, P]
        L.or_exact_cost_parts.argtypes = [i32, P, P, P, P, f64, P]
        L.or_grid_rule.argtypes = [i32, P, f32, i32, i32, i32, P, P]
        L.or_spread.argtypes = [i32, P, P, P, i32, P, P]
        L.or_conv_direct.argtypes = [i32, f64, f64, P, P]
        L.or_gather.argtypes = [i32, P, P, P, i32, P, P]
        L.or_attractive.argtypes = [i32, P, P, P, P, P]
        L.or_exact_rows.argtypes = [i32, P, P, P, P, f64, i32, P, P, P, P]
        L.or_exact_z.argtypes = [i32, P, P]
        L.or_exact_cost_step.argtypes = [i32, P, P, P, P, f64, i32, i32, f64, P]
        L.or_set_threads.argtypes = [i32]
        L.or_set_threads.restype = i32
        _lib = L
    return _lib


def set_threads(t: int = 0) -> int:
    """Threads of the oracle's row-parallel loops (t <= 0 leaves the count
    unchanged); returns the count in use."""
    return int(lib().or_set_threads(int(t)))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# --------------------------------------------------------------------------
# C0 (Alg. 3, preprocessing): partial BFS, perplexity calibration, Eq. 2.
# --------------------------------------------------------------------------
def k_from_perplexity(u: float) -> int:
    """k = 3u (Sec. 3.1); reading for fractional u: k = ceil(3u)."""
    return int(math.ceil(3.0 * u - 1e-9))


def partial_bfs(row_ptr, col, k: int, s0: int = 0, s1: int | None = None):
    """Partial BFS from every source in [s0, s1) (Sec. 3.1).  Returns
    (nbr int32[(s1-s0), k], hop int32[...], cnt int32[s1-s0])."""
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    n = row_ptr.shape[0] - 1
    s1 = n if s1 is None else s1
    rows = s1 - s0
    nbr = np.empty((rows, k), np.int32)
    hop = np.empty((rows, k), np.int32)
    cnt = np.empty(rows, np.int32)
    rc = lib().or_partial_bfs(n, _p(row_ptr), _p(col), k, s0, s1, _p(nbr), _p(hop), _p(cnt))
    if rc != 0:
        raise ValueError(f"or_partial_bfs failed ({rc})")
    return nbr, hop, cnt


def calibrate(hop, cnt, perplexity: float, tol: float = 1e-5, max_steps: int = 100):
    """Per-row beta search (Eq. 3, perplexity definition of Sec. 2.1).
    Returns (beta f64[n], pcond f64[n, k], converged u8[n])."""
    hop = _c(hop, np.int32)
    cnt = _c(cnt, np.int32)
    n, k = hop.shape
    beta = np.empty(n, np.float64)
    pcond = np.empty((n, k), np.float64)
    conv = np.empty(n, np.uint8)
    rc = lib().or_calibrate(n, k, _p(hop), _p(cnt), float(perplexity), float(tol), int(max_steps),
                            _p(beta), _p(pcond), _p(conv))
    if rc != 0:
        raise ValueError(f"or_calibrate failed ({rc})")
    return beta, pcond, conv


def symmetrize(nbr, cnt, pcond):
    """Eq. 2: P = (Pc + Pc^T)/(2n) over the union of supports, CSR with
    ascending columns.  Returns (P_row int64, P_col int32, P_val f64)."""
    nbr = _c(nbr, np.int32)
    cnt = _c(cnt, np.int32)
    pcond = _c(pcond, np.float64)
    n, k = nbr.shape
    cap = max(1, 2 * int(cnt.sum()))
    P_row = np.empty(n + 1, np.int64)
    P_col = np.empty(cap, np.int32)
    P_val = np.empty(cap, np.float64)
    nnz = lib().or_symmetrize(n, k, _p(nbr), _p(cnt), _p(pcond), _p(P_row), _p(P_col), _p(P_val), cap)
    if nnz < 0:
        raise ValueError(f"or_symmetrize failed ({nnz})")
    return P_row, P_col[:nnz].copy(), P_val[:nnz].copy()


@dataclass
class Affinities:
    nbr: np.ndarray
    hop: np.ndarray
    cnt: np.ndarray
    beta: np.ndarray
    pcond: np.ndarray
    converged: np.ndarray
    P_row: np.ndarray
    P_col: np.ndarray
    P_val64: np.ndarray

    @property
    def P_val32(self) -> np.ndarray:
        return self.P_val64.astype(np.float32)


def preprocess(row_ptr, col, perplexity: float, tol: float = 1e-5, max_steps: int = 100) -> Affinities:
    """C0 of Alg. 3: partial BFS with k = 3u, calibration, symmetrisation."""
    k = k_from_perplexity(perplexity)
    nbr, hop, cnt = partial_bfs(row_ptr, col, k)
    beta, pcond, conv = calibrate(hop, cnt, perplexity, tol, max_steps)
    P_row, P_col, P_val = symmetrize(nbr, cnt, pcond)
    return Affinities(nbr, hop, cnt, beta, pcond, conv, P_row, P_col, P_val)


# --------------------------------------------------------------------------
# Loop terms.
# --------------------------------------------------------------------------
@dataclass
class Stage:
    """Per-stage multipliers (Sec. 2.1: lambda_KL, lambda_c, lambda_r change
    per descent stage; values not given in the paper)."""
    iters: int = 250
    lambda_kl: float = 1.0
    lambda_c: float = 1.2
    lambda_r: float = 0.0
    exaggeration: float = 1.0
    momentum: float = 0.5


def default_stages(total_iters: int = 1000) -> list[Stage]:
    """Reading (parity unpinned): stage 1 = 250 iterations with
    (lambda_KL, lambda_c, lambda_r) = (1, 1.2, 0), momentum 0.5; stage 2 = the
    rest with (1, 0.01, 0.6), momentum 0.8."""
    first = min(250, total_iters)
    st = [Stage(first, 1.0, 1.2, 0.0, 1.0, 0.5)]
    if total_iters > first:
        st.append(Stage(total_iters - first, 1.0, 0.01, 0.6, 1.0, 0.8))
    return st


@dataclass
class GridParams:
    """Interpolation grid rule (Sec. 2.3: I intervals, P nodes per interval;
    constants not in the paper)."""
    nodes_per_box: int = 3
    box_width_max: float = 0.25
    min_boxes: int = 50
    max_boxes: int = 1350
    eps: float = EPS_DEFAULT


def as_csr64(P_row, P_col, P_val):
    return _c(P_row, np.int64), _c(P_col, np.int32), _c(P_val, np.float64)


def exact_sums(Y, P_row, P_col, P_val, eps: float = EPS_DEFAULT):
    """O(n^2) sums A, R, E and Z (Eq. 6 split, Sec. 3.3 kernel).  Y (n,2)."""
    Y = _c(Y, np.float64)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    n = Y.shape[0]
    A = np.empty((n, 2)); R = np.empty((n, 2)); E = np.empty((n, 2)); Z = np.zeros(1)
    lib().or_exact_sums(n, _p(Y), _p(P_row), _p(P_col), _p(P_val), float(eps), _p(A), _p(R), _p(E), _p(Z))
    return A, R, E, float(Z[0])


def exact_rows(Y, P_row, P_col, P_val, rows, eps: float = EPS_DEFAULT):
    """The O(n^2) sums A, R, E of exact_sums for the target rows ``rows``
    only (each over every source); Z is not included (exact_z)."""
    Y = _c(Y, np.float64)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    rows = _c(rows, np.int32)
    m = rows.shape[0]
    A = np.empty((m, 2)); R = np.empty((m, 2)); E = np.empty((m, 2))
    if lib().or_exact_rows(Y.shape[0], _p(Y), _p(P_row), _p(P_col), _p(P_val), float(eps), m, _p(rows),
                           _p(A), _p(R), _p(E)) != 0:
        raise ValueError("or_exact_rows: row out of range")
    return A, R, E


def exact_z(Y) -> float:
    """Z = sum_{i != j} 1/(1 + d_ij^2) over all ordered pairs."""
    Y = _c(Y, np.float64)
    z = np.zeros(1)
    if lib().or_exact_z(Y.shape[0], _p(Y), _p(z)) != 0:
        raise MemoryError("or_exact_z")
    return float(z[0])


def exact_cost_central_difference(Y, P_row, P_col, P_val, st: Stage, i: int, d: int, h: float, Z: float,
                                  eps: float = EPS_DEFAULT) -> float:
    """(C(Y + h e_id) - C(Y - h e_id)) / 2h for the exact cost of exact_cost
    (Eq. 1, entropy reading), from only the terms that involve vertex i;
    Z = exact_z(Y) and S = sum of P_val are the unperturbed values."""
    Y = _c(Y, np.float64)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    n = Y.shape[0]
    o = np.zeros(5)
    if lib().or_exact_cost_step(n, _p(Y), _p(P_row), _p(P_col), _p(P_val), float(eps), int(i), int(d), float(h),
                                _p(o)) != 0:
        raise ValueError("or_exact_cost_step: bad coordinate")
    S = float(np.sum(P_val))
    # ln(Z + o1) - ln(Z + o2) as one log1p: the two logarithms of numbers near
    # Z would cancel to a few ulps of ln Z
    dc = (st.lambda_kl * (o[0] + S * math.log1p((o[1] - o[2]) / (Z + o[2])))
          + st.lambda_c / (2.0 * n) * o[4] - st.lambda_r / (4.0 * n * n) * o[3])
    return dc / (2.0 * h)


def assemble(Y, A, R, E, Z: float, S: float, st: Stage, n: int):
    """dC/dX_i = 4 l_KL (alpha A_i - (S/Z) R_i) + (l_c/n) X_i - (l_r/n^2) E_i.
    Eq. 6 (scaled by lambda_KL, Eq. 1) with S = sum p (= 1 for normalised P);
    compression from Eq. 1; entropy from Sec. 3.3 with the sign reading that
    makes it repulsive (moving against the gradient pushes points apart)."""
    Y = np.asarray(Y, np.float64)
    return (4.0 * st.lambda_kl * (st.exaggeration * A - (S / Z) * R)
            + (st.lambda_c / n) * Y - (st.lambda_r / (n * n)) * E)


def exact_gradient(Y, P_row, P_col, P_val, st: Stage, eps: float = EPS_DEFAULT):
    A, R, E, Z = exact_sums(Y, P_row, P_col, P_val, eps)
    S = float(np.sum(np.asarray(P_val, np.float64)))
    n = np.asarray(Y).shape[0]
    return assemble(Y, A, R, E, Z, S, st, n), dict(A=A, R=R, E=E, Z=Z, S=S)


def exact_cost(Y, P_row, P_col, P_val, st: Stage, eps: float = EPS_DEFAULT, literal: bool = False):
    """C = l_KL [sum p ln p + sum p ln(1+d^2) + S ln Z] + (l_c/2n) sum |X|^2
         - (l_r/4n^2) sum_{i!=j} ln(eps + d^2)
    (Eq. 1 with Eq. 4 and q_ij; the entropy term in the eps-regularised
    reading whose gradient is the Sec. 3.3 kernel).  ``literal=True`` uses the
    paper's -(l_r/2n^2) sum ln(|d|) instead (eps = 0 only)."""
    Y = _c(Y, np.float64)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    n = Y.shape[0]
    out = np.zeros(7)
    lib().or_exact_cost_parts(n, _p(Y), _p(P_row), _p(P_col), _p(P_val), float(eps), _p(out))
    plogp, plogk, Z, sq, lent, llit, S = out
    ckl = st.lambda_kl * (plogp + plogk + S * math.log(Z))
    ccmp = st.lambda_c / (2.0 * n) * sq
    cent = -(st.lambda_r / (2.0 * n * n)) * llit if literal else -(st.lambda_r / (4.0 * n * n)) * lent
    return ckl + ccmp + cent, dict(kl=ckl, cmp=ccmp, ent=cent, Z=Z, S=S)


def grad_pvals(Y, P_row, P_col, P_val, st: Stage, eps: float = EPS_DEFAULT):
    """dC/dp_e = l_KL (ln p_e + 1 + ln(1 + d_e^2) + ln Z), each stored entry an
    independent leaf (derivative of the exact cost above)."""
    Y = np.asarray(Y, np.float64)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    n = Y.shape[0]
    _, parts = exact_cost(Y, P_row, P_col, P_val, st, eps)
    rows = np.repeat(np.arange(n), np.diff(P_row))
    d2 = np.sum((Y[rows] - Y[P_col]) ** 2, axis=1)
    with np.errstate(divide="ignore"):  # p_e = 0 gives -inf, the derivative's limit
        lnp = np.log(P_val)
    return st.lambda_kl * (lnp + 1.0 + np.log1p(d2) + math.log(parts["Z"]))


# ---- INTERP (Sec. 2.3 + Sec. 3.3) ----------------------------------------
@dataclass
class GridInfo:
    lo: float
    hi: float
    ext: float
    h: float
    s: float
    centre: float
    I: int
    M: int
    raw_f: np.ndarray = field(repr=False)
    raw_i: np.ndarray = field(repr=False)


def grid_rule(Y32, gp: GridParams) -> GridInfo:
    """FP32 grid decisions: lo/hi = min/max over all coordinates, I =
    max(min_boxes, ceil(ext / box_width_max)) rounded up to a 5-smooth size,
    h = ext / I, node spacing s = h / P."""
    Y32 = _c(Y32, np.float32)
    g = np.zeros(6, np.float32)
    ig = np.zeros(2, np.int32)
    rc = lib().or_grid_rule(Y32.shape[0], _p(Y32), float(gp.box_width_max), gp.min_boxes,
                            gp.max_boxes, gp.nodes_per_box, _p(g), _p(ig))
    if rc != 0:
        raise ValueError("or_grid_rule failed")
    return GridInfo(float(g[0]), float(g[1]), float(g[2]), float(g[3]), float(g[4]), float(g[5]),
                    int(ig[0]), int(ig[1]), g, ig)


def spread(Y32, gi: GridInfo, P: int):
    """W (4, M, M): charges (1, x~, y~, x~^2+y~^2) spread with Lagrange weights."""
    Y32 = _c(Y32, np.float32)
    W = np.empty((4, gi.M, gi.M))
    box = np.empty((Y32.shape[0], 2), np.int32)
    lib().or_spread(Y32.shape[0], _p(Y32), _p(gi.raw_f), _p(gi.raw_i), P, _p(W), _p(box))
    return W, box


def kernel_values(M: int, s: float, eps: float):
    """K2 and Ke at node offsets (dx, dy) in [0, M)^2 (both even in dx, dy)."""
    d = np.arange(M) * s
    d2 = d[None, :] ** 2 + d[:, None] ** 2
    k1 = 1.0 / (1.0 + d2)
    return k1 * k1, 1.0 / (eps + d2)


def conv_direct(W, s: float, eps: float):
    W = _c(W, np.float64)
    M = W.shape[1]
    out = np.empty((7, M, M))
    lib().or_conv_direct(M, float(s), float(eps), _p(W), _p(out))
    return out


def conv_fft(W, s: float, eps: float):
    """Same sums as conv_direct via a zero-padded 2M x 2M circulant embedding
    and numpy's FP64 FFT."""
    W = np.asarray(W, np.float64)
    M = W.shape[1]
    L = 2 * M
    k2, ke = kernel_values(M, s, eps)

    def embed(kv):
        c = np.zeros((L, L))
        c[:M, :M] = kv
        c[L - M + 1:, :M] = kv[1:][::-1, :]
        c[:M, L - M + 1:] = kv[:, 1:][:, ::-1]
        c[L - M + 1:, L - M + 1:] = kv[1:, 1:][::-1, ::-1]
        return np.fft.rfft2(c)

    K2h, Keh = embed(k2), embed(ke)
    out = np.empty((7, M, M))
    for ch in range(4):
        Wh = np.fft.rfft2(W[ch], s=(L, L))
        out[ch] = np.fft.irfft2(Wh * K2h, s=(L, L))[:M, :M]
        if ch < 3:
            out[4 + ch] = np.fft.irfft2(Wh * Keh, s=(L, L))[:M, :M]
    return out


def gather(Y32, gi: GridInfo, P: int, fld):
    Y32 = _c(Y32, np.float32)
    fld = _c(fld, np.float64)
    Phi = np.empty((Y32.shape[0], 7))
    lib().or_gather(Y32.shape[0], _p(Y32), _p(gi.raw_f), _p(gi.raw_i), P, _p(fld), _p(Phi))
    return Phi


def attractive(Y32, P_row, P_col, P_val):
    Y32 = _c(Y32, np.float32)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    A = np.empty((Y32.shape[0], 2))
    lib().or_attractive(Y32.shape[0], _p(Y32), _p(P_row), _p(P_col), _p(P_val), _p(A))
    return A


def interp_fields(Y32, gp: GridParams, conv: str = "auto"):
    """Grid rule, spread, convolution and gather.  Returns (Phi (n,7), W,
    fields (7,M,M), GridInfo)."""
    gi = grid_rule(Y32, gp)
    W, _ = spread(Y32, gi, gp.nodes_per_box)
    if conv == "direct" or (conv == "auto" and gi.M <= 48):
        fld = conv_direct(W, gi.s, gp.eps)
    else:
        fld = conv_fft(W, gi.s, gp.eps)
    return gather(Y32, gi, gp.nodes_per_box, fld), W, fld, gi


def z_from_points(Y32, Phi, centre: float):
    """Z = sum_i [(1+x~^2+y~^2) Phi0 - 2x~ Phi1 - 2y~ Phi2 + Phi3] - n: the
    K2 sums times (1 + d^2) give the K1 sums (Sec. 2.3); the self terms
    K1(0) = 1 are removed."""
    Y = np.asarray(Y32, np.float64) - centre
    x, y = Y[:, 0], Y[:, 1]
    return float(np.sum((1 + x * x + y * y) * Phi[:, 0] - 2 * x * Phi[:, 1] - 2 * y * Phi[:, 2]
                        + Phi[:, 3]) - Y.shape[0])


def z_from_grid(W, fld, n: int):
    """The same Z as a sum over grid nodes (gather is the transpose of spread):
    sum_t [phi0 (W0 + W3) - 2 phi1 W1 - 2 phi2 W2 + phi3 W0] - n."""
    return float(np.sum(fld[0] * (W[0] + W[3]) - 2 * fld[1] * W[1] - 2 * fld[2] * W[2] + fld[3] * W[0])
                 - n)


def log_kernel_sum(W0, s: float, eps: float):
    """sum_t W0[t] (K_ln * W0)[t] with K_ln = ln(eps + d^2) at node offsets:
    the double sum sum_{i,j} ln(eps + d_ij^2) with the kernel interpolated in
    both arguments (spread of charge 1, W0), self terms included.  By a
    zero-padded circulant embedding and numpy's FP64 FFT."""
    W0 = np.asarray(W0, np.float64)
    M = W0.shape[0]
    L = 2 * M
    d = np.arange(M) * s
    kl = np.log(eps + d[None, :] ** 2 + d[:, None] ** 2)
    c = np.zeros((L, L))
    c[:M, :M] = kl
    c[L - M + 1:, :M] = kl[1:][::-1, :]
    c[:M, L - M + 1:] = kl[:, 1:][:, ::-1]
    c[L - M + 1:, L - M + 1:] = kl[1:, 1:][::-1, ::-1]
    conv = np.fft.irfft2(np.fft.rfft2(W0, s=(L, L)) * np.fft.rfft2(c), s=(L, L))[:M, :M]
    return float(np.sum(W0 * conv))


def log_kernel_sum_direct(W0, s: float, eps: float):
    """The same double sum over node pairs, directly (small grids)."""
    W0 = np.asarray(W0, np.float64)
    M = W0.shape[0]
    t = np.arange(M)
    tot = 0.0
    for ay in range(M):
        for ax in range(M):
            if W0[ay, ax] == 0.0:
                continue
            d2 = ((t[:, None] - ay) ** 2 + (t[None, :] - ax) ** 2) * (s * s)
            tot += W0[ay, ax] * float(np.sum(W0 * np.log(eps + d2)))
    return tot


def interp_cost(Y32, P_row, P_col, P_val, st: Stage, gp: GridParams):
    """The cost with the GPU's interpolation: exact sparse KL sums, Z from
    the grid, and the entropy double sum from log_kernel_sum minus the n
    self terms ln(eps).  Returns dict(kl, cmp, ent, total, Z, S, lsum)."""
    Y32 = _c(Y32, np.float32)
    n = Y32.shape[0]
    Phi, W, fld, gi = interp_fields(Y32, gp)
    Z = z_from_points(Y32, Phi, gi.centre)
    lsum = log_kernel_sum(W[0], gi.s, gp.eps)
    Y = Y32.astype(np.float64)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    rows = np.repeat(np.arange(n), np.diff(P_row))
    d2 = np.sum((Y[rows] - Y[P_col]) ** 2, axis=1)
    pos = P_val > 0
    plogp = float(np.sum(P_val[pos] * np.log(P_val[pos])))
    plogk = float(np.sum(P_val * np.log1p(d2)))
    S = float(np.sum(P_val))
    kl = st.lambda_kl * (plogp + plogk + S * math.log(Z))
    cmp = st.lambda_c / (2.0 * n) * float(np.sum(Y * Y))
    ent = -(st.lambda_r / (4.0 * n * n)) * (lsum - n * math.log(gp.eps))
    return dict(kl=kl, cmp=cmp, ent=ent, total=kl + cmp + ent, Z=Z, S=S, lsum=lsum)


def interp_gradient(Y32, P_row, P_col, P_val, st: Stage, gp: GridParams, conv: str = "auto"):
    """Per-iteration L-tsNET gradient with the same interpolation as the GPU
    path: exact sparse attraction plus interpolated repulsion, Z and entropy.
    Returns (grad (n,2), parts dict)."""
    Y32 = _c(Y32, np.float32)
    n = Y32.shape[0]
    Phi, W, fld, gi = interp_fields(Y32, gp, conv)
    A = attractive(Y32, P_row, P_col, P_val)
    Yt = Y32.astype(np.float64) - gi.centre
    Z = z_from_points(Y32, Phi, gi.centre)
    R = np.stack([Yt[:, 0] * Phi[:, 0] - Phi[:, 1], Yt[:, 1] * Phi[:, 0] - Phi[:, 2]], axis=1)
    E = np.stack([Yt[:, 0] * Phi[:, 4] - Phi[:, 5], Yt[:, 1] * Phi[:, 4] - Phi[:, 6]], axis=1)
    S = float(np.sum(np.asarray(P_val, np.float64)))
    g = assemble(Y32, A, R, E, Z, S, st, n)
    return g, dict(A=A, R=R, E=E, Z=Z, S=S, grid=gi, Phi=Phi, W=W, fields=fld)


def interp_grad_pvals(Y32, P_row, P_col, P_val, st: Stage, gp: GridParams):
    """dC/dp_e of interp_cost, each stored entry an independent leaf:
    l_KL (ln p_e + 1 + ln(1 + d_e^2) + ln Z) with Z from the grid (Z does not
    depend on P, so this is grad_pvals with the interpolated Z)."""
    Y32 = _c(Y32, np.float32)
    P_row, P_col, P_val = as_csr64(P_row, P_col, P_val)
    n = Y32.shape[0]
    Phi, _, _, gi = interp_fields(Y32, gp)
    Z = z_from_points(Y32, Phi, gi.centre)
    Y = Y32.astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(P_row))
    d2 = np.sum((Y[rows] - Y[P_col]) ** 2, axis=1)
    with np.errstate(divide="ignore"):  # p_e = 0 gives -inf, the derivative's limit
        lnp = np.log(P_val)
    return st.lambda_kl * (lnp + 1.0 + np.log1p(d2) + math.log(Z))


def update(Y, upd, gains, grad, momentum: float, lr: float):
    """Gradient step with momentum and gains (reading: the t-SNE optimiser of
    van der Maaten and Hinton; parity unpinned): a gain grows by 0.2 where the
    gradient's sign differs from the previous step's, else shrinks by x0.8,
    floored at 0.01; step = momentum*step - lr*gain*grad; Y += step."""
    flip = np.sign(grad) != np.sign(upd)
    gains = np.where(flip, gains + 0.2, gains * 0.8)
    gains = np.maximum(gains, 0.01)
    upd = momentum * upd - lr * gains * grad
    return Y + upd, upd, gains


def auto_learning_rate(n: int) -> float:
    return max(200.0, n / 12.0)


def run(Y0, P_row, P_col, P_val, stages: list[Stage], gp: GridParams, lr: float = 0.0,
        iters: int | None = None, exact: bool = False, keep_fp32: bool = True):
    """Alg. 3 loop: the gradient (interpolated, or exact O(n^2)) followed by the
    update, over the stage schedule.  The layout is kept in FP32 between
    iterations when ``keep_fp32`` (the grid decisions need FP32 input)."""
    n = Y0.shape[0]
    lr = lr if lr > 0 else auto_learning_rate(n)
    Y = np.asarray(Y0, np.float64).copy()
    upd = np.zeros_like(Y)
    gains = np.ones_like(Y)
    sched = []
    for st in stages:
        sched += [st] * st.iters
    if iters is not None:
        sched = sched[:iters]
    for st in sched:
        Y32 = Y.astype(np.float32)
        if exact:
            g, _ = exact_gradient(Y32.astype(np.float64) if keep_fp32 else Y, P_row, P_col, P_val, st, gp.eps)
        else:
            g, _ = interp_gradient(Y32, P_row, P_col, P_val, st, gp)
        Y, upd, gains = update(Y32.astype(np.float64) if keep_fp32 else Y, upd, gains, g, st.momentum, lr)
    return Y
