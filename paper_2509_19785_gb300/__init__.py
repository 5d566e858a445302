"""GB300 L-tsNET: Python binding of libltsnet.so (include/ltsnet.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory (including the workspaces the
library asks for) and the current CUDA stream.  There is no CPU fallback: if
the library is missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libltsnet.so")

OK = 0
WARN_NOT_CONVERGED = 1
ERR_BAD_GRAPH = -6
ERR_NONFINITE = -5
FLAG_PLAIN = 1
FLAG_NO_REORDER = 2
CONV_FFT = 0
CONV_DFT_GEMM = 1
MAX_K = 4096
KERNEL_FUSED_UPDATE, KERNEL_SPREAD, KERNEL_CONV = 1, 2, 3

# Every entry point declared in include/ltsnet.h.
ABI_SYMBOLS = (
    "ltsnet_default_params", "ltsnet_default_stages", "ltsnet_status_string", "ltsnet_last_cuda_error",
    "ltsnet_poll_status",
    "ltsnet_knn_bfs", "ltsnet_calibrate", "ltsnet_symmetrize_max_nnz", "ltsnet_symmetrize_workspace_size",
    "ltsnet_symmetrize", "ltsnet_symmetrize_static_max_entries", "ltsnet_symmetrize_static",
    "ltsnet_bfs_order_workspace_size", "ltsnet_bfs_order", "ltsnet_gradient_workspace_size", "ltsnet_gradient",
    "ltsnet_cost", "ltsnet_grad_pvals", "ltsnet_optimize_workspace_size",
    "ltsnet_optimize", "ltsnet_run_workspace_size", "ltsnet_run", "ltsnet_run_host",
    "ltsnet_run_batched_workspace_size", "ltsnet_run_batched", "ltsnet_launch_count",
    "ltsnet_profile_begin", "ltsnet_profile_end", "ltsnet_pivot_mds_workspace_size", "ltsnet_pivot_mds",
    "ltsnet_quality_workspace_size", "ltsnet_neighbourhood_preservation", "ltsnet_stress",
    "ltsnet_gradient_quadtree_workspace_size", "ltsnet_gradient_quadtree",
    "ltsnet_optimize_quadtree_workspace_size", "ltsnet_optimize_quadtree",
)


class LtsnetError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {status_string(code)} ({code})"
        if code == -3:
            msg += f": {lib().ltsnet_last_cuda_error().decode()}"
        super().__init__(msg)


class CStage(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("lambda_kl", ctypes.c_float), ("lambda_c", ctypes.c_float),
                ("lambda_r", ctypes.c_float), ("exaggeration", ctypes.c_float), ("momentum", ctypes.c_float)]


class CParams(ctypes.Structure):
    _fields_ = [("perplexity", ctypes.c_float), ("eps", ctypes.c_float), ("nodes_per_box", ctypes.c_int32),
                ("box_width_max", ctypes.c_float), ("min_boxes", ctypes.c_int32), ("max_boxes", ctypes.c_int32),
                ("learning_rate", ctypes.c_float), ("beta_max_steps", ctypes.c_int32), ("beta_tol", ctypes.c_double),
                ("n_stages", ctypes.c_int32), ("stages", ctypes.POINTER(CStage)), ("flags", ctypes.c_int32),
                ("conv_mode", ctypes.c_int32)]


class CBatchConfig(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("n_workers", ctypes.c_int32), ("fft_blocks", ctypes.c_int32),
                ("spread_blocks", ctypes.c_int32), ("max_boxes_used", ctypes.c_void_p),
                ("max_boxes", ctypes.c_void_p)]


BATCH_ONE_LAUNCH = 0
BATCH_PER_GRAPH = 1

_lib = None


def lib():
    """Load libltsnet.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libltsnet.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, f64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        pp = ctypes.POINTER(CParams)
        L.ltsnet_default_params.restype = CParams
        L.ltsnet_default_stages.argtypes = [i32, ctypes.POINTER(CStage)]
        L.ltsnet_default_stages.restype = i32
        L.ltsnet_status_string.argtypes = [i32]
        L.ltsnet_status_string.restype = ctypes.c_char_p
        L.ltsnet_last_cuda_error.restype = ctypes.c_char_p
        L.ltsnet_poll_status.argtypes = [P, sz, P]
        L.ltsnet_knn_bfs.argtypes = [P, P, i32, i32, P, P, P, P, sz, P]
        L.ltsnet_calibrate.argtypes = [P, P, i32, i32, f64, f64, i32, P, P, P, P]
        L.ltsnet_symmetrize_max_nnz.argtypes = [i32, i32]
        L.ltsnet_symmetrize_max_nnz.restype = i64
        L.ltsnet_symmetrize_workspace_size.argtypes = [i32, i32]
        L.ltsnet_symmetrize_workspace_size.restype = sz
        L.ltsnet_symmetrize.argtypes = [P, P, P, i32, i32, P, P, P, i64, ctypes.POINTER(i64), P, sz, P]
        L.ltsnet_symmetrize_static_max_entries.restype = i64
        L.ltsnet_symmetrize_static.argtypes = [P, P, P, i32, i32, P, P, P, i64, ctypes.POINTER(i64), P]
        L.ltsnet_bfs_order_workspace_size.argtypes = [i32]
        L.ltsnet_bfs_order_workspace_size.restype = sz
        L.ltsnet_bfs_order.argtypes = [P, P, i32, P, P, ctypes.POINTER(i32), P, sz, P]
        L.ltsnet_gradient_workspace_size.argtypes = [i32, pp]
        L.ltsnet_gradient_workspace_size.restype = sz
        L.ltsnet_gradient.argtypes = [P, P, P, i32, P, ctypes.POINTER(CStage), pp, P, P, P, P, sz, P]
        L.ltsnet_cost.argtypes = [P, P, P, i32, P, ctypes.POINTER(CStage), pp, P, P, P, sz, P]
        L.ltsnet_grad_pvals.argtypes = [P, P, P, i32, P, ctypes.POINTER(CStage), pp, P, P, sz, P]
        L.ltsnet_optimize_workspace_size.argtypes = [i32, pp]
        L.ltsnet_optimize_workspace_size.restype = sz
        L.ltsnet_optimize.argtypes = [P, P, P, i32, pp, P, P, P, i32, i32, P, sz, P]
        L.ltsnet_run_workspace_size.argtypes = [i32, i64, pp]
        L.ltsnet_run_workspace_size.restype = sz
        L.ltsnet_run.argtypes = [P, P, i32, pp, P, P, sz, P]
        L.ltsnet_run_host.argtypes = [P, P, i32, pp, P, P, sz, P]
        bc = ctypes.POINTER(CBatchConfig)
        L.ltsnet_run_batched_workspace_size.argtypes = [i32, P, P, pp, bc]
        L.ltsnet_run_batched_workspace_size.restype = sz
        L.ltsnet_run_batched.argtypes = [i32, P, P, P, P, pp, P, P, sz, bc, P]
        L.ltsnet_pivot_mds_workspace_size.argtypes = [i32, i32]
        L.ltsnet_pivot_mds_workspace_size.restype = sz
        L.ltsnet_pivot_mds.argtypes = [P, P, i32, i32, i32, f64, P, P, P, ctypes.POINTER(f64), P, sz, P]
        L.ltsnet_pivot_mds.restype = i32
        L.ltsnet_quality_workspace_size.argtypes = [i32, i64]
        L.ltsnet_quality_workspace_size.restype = sz
        L.ltsnet_neighbourhood_preservation.argtypes = [P, P, i32, P, P, P, ctypes.POINTER(f64), P, sz, P]
        L.ltsnet_neighbourhood_preservation.restype = i32
        L.ltsnet_stress.argtypes = [P, P, i32, P, P, i32, ctypes.POINTER(f64), P, sz, P]
        L.ltsnet_stress.restype = i32
        L.ltsnet_gradient_quadtree_workspace_size.argtypes = [i32, pp, i32]
        L.ltsnet_gradient_quadtree_workspace_size.restype = sz
        L.ltsnet_gradient_quadtree.argtypes = [P, P, P, i32, P, ctypes.POINTER(CStage), pp, ctypes.c_float, i32, P, P,
                                               ctypes.POINTER(f64), P, sz, P]
        L.ltsnet_gradient_quadtree.restype = i32
        L.ltsnet_optimize_quadtree_workspace_size.argtypes = [i32, pp, i32]
        L.ltsnet_optimize_quadtree_workspace_size.restype = sz
        L.ltsnet_optimize_quadtree.argtypes = [P, P, P, i32, pp, ctypes.c_float, i32, P, P, P, i32, i32, P, sz, P]
        L.ltsnet_optimize_quadtree.restype = i32
        L.ltsnet_launch_count.restype = i64
        L.ltsnet_profile_begin.argtypes = [i32, i32]
        L.ltsnet_profile_end.argtypes = [i32, ctypes.POINTER(f64), ctypes.POINTER(i32)]
        for name in ("ltsnet_poll_status", "ltsnet_knn_bfs", "ltsnet_calibrate", "ltsnet_symmetrize",
                     "ltsnet_symmetrize_static", "ltsnet_bfs_order",
                     "ltsnet_gradient", "ltsnet_optimize", "ltsnet_run", "ltsnet_run_host",
                     "ltsnet_profile_begin", "ltsnet_profile_end"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().ltsnet_status_string(int(code)).decode()


def _check(rc: int, what: str, allow_warn: bool = True) -> int:
    if rc < 0 or (rc > 0 and not allow_warn):
        raise LtsnetError(rc, what)
    return rc


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
@dataclass
class Stage:
    """One descent stage: the multipliers of the three cost terms (Eq. 1),
    exaggeration of P in the attraction, optimiser momentum."""
    iters: int
    lambda_kl: float = 1.0
    lambda_c: float = 1.2
    lambda_r: float = 0.0
    exaggeration: float = 1.0
    momentum: float = 0.5

    def to_c(self) -> CStage:
        return CStage(int(self.iters), self.lambda_kl, self.lambda_c, self.lambda_r, self.exaggeration, self.momentum)


def default_stages(total_iters: int = 1000) -> list[Stage]:
    buf = (CStage * 2)()
    k = lib().ltsnet_default_stages(int(total_iters), buf)
    return [Stage(b.iters, b.lambda_kl, b.lambda_c, b.lambda_r, b.exaggeration, b.momentum) for b in buf[:k]]


@dataclass
class Params:
    perplexity: float = 30.0
    eps: float = 1.0 / 20.0
    nodes_per_box: int = 3
    box_width_max: float = 0.25
    min_boxes: int = 50
    max_boxes: int = 640
    learning_rate: float = 0.0
    beta_max_steps: int = 100
    beta_tol: float = 1e-5
    stages: list = field(default_factory=lambda: None)
    plain: bool = False
    reorder: bool = True
    conv_mode: int = 0  # 0: FP32 FFT; 1: split-BF16 DFT matrix products on the tensor cores

    @property
    def k(self) -> int:
        return int(math.ceil(3.0 * self.perplexity - 1e-9))

    def schedule(self) -> list[Stage]:
        return self.stages if self.stages is not None else default_stages(1000)

    def to_c(self):
        st = self.schedule()
        arr = (CStage * max(1, len(st)))(*[s.to_c() for s in st])
        p = CParams(self.perplexity, self.eps, self.nodes_per_box, self.box_width_max, self.min_boxes,
                    self.max_boxes, self.learning_rate, self.beta_max_steps, self.beta_tol, len(st),
                    ctypes.cast(arr, ctypes.POINTER(CStage)),
                    (FLAG_PLAIN if self.plain else 0) | (0 if self.reorder else FLAG_NO_REORDER),
                    int(self.conv_mode))
        p._keep = arr  # keep the stage array alive with the struct
        return p


# --------------------------------------------------------------------------
# torch plumbing
# --------------------------------------------------------------------------
def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (no CPU fallback)")
    return torch


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None) -> ctypes.c_void_p:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device=None):
    torch = _torch()
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def _dev(t, dtype):
    torch = _torch()
    t = torch.as_tensor(t)
    return t.to(device="cuda", dtype=dtype).contiguous()


def knn_bfs(row_ptr, col, k: int):
    """Partial BFS neighbours (Sec. 3.1).  Returns (nbr int32 [n,k], hop
    uint16 [n,k], cnt int32 [n]) on the GPU."""
    torch = _torch()
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    n = row_ptr.numel() - 1
    nbr = torch.empty((n, k), dtype=torch.int32, device="cuda")
    hop = torch.empty((n, k), dtype=torch.uint16, device="cuda")
    cnt = torch.empty((n,), dtype=torch.int32, device="cuda")
    ws = _workspace(256)
    ws.zero_()
    _check(lib().ltsnet_knn_bfs(_ptr(row_ptr), _ptr(col), n, k, _ptr(nbr), _ptr(hop), _ptr(cnt), _ptr(ws),
                                ws.numel(), _stream()), "ltsnet_knn_bfs")
    _check(lib().ltsnet_poll_status(_ptr(ws), ws.numel(), _stream()), "ltsnet_knn_bfs (device)")
    return nbr, hop, cnt


def pivot_mds_workspace(n: int, n_pivots: int):
    """Workspace for ltsnet_pivot_mds (device bytes)."""
    nb = lib().ltsnet_pivot_mds_workspace_size(int(n), int(n_pivots))
    if nb == 0:
        raise LtsnetError(-1, "ltsnet_pivot_mds_workspace_size")
    return _workspace(nb)


def pivot_mds(row_ptr, col, n_pivots: int = 100, first: int = 0, init_std: float = 1e-4, ws=None,
              return_dist: bool = False):
    """Pivot MDS initial layout (the first step of Alg. 1-3).  Returns
    (Y f32 [n,2], pivots int32 [k], eigvals (sigma_1^2, sigma_2^2)) on the GPU,
    plus the distance rows uint16 [k,n] (0xFFFF = unreached) if
    return_dist."""
    torch = _torch()
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    n = row_ptr.numel() - 1
    k = int(n_pivots)
    if ws is None:
        ws = pivot_mds_workspace(n, k)
    Y = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    piv = torch.empty((k,), dtype=torch.int32, device="cuda")
    dist = torch.empty((k, n), dtype=torch.uint16, device="cuda") if return_dist else None
    eig = (ctypes.c_double * 2)()
    _check(lib().ltsnet_pivot_mds(_ptr(row_ptr), _ptr(col), n, k, int(first), float(init_std), _ptr(Y), _ptr(piv),
                                  _ptr(dist), eig, _ptr(ws), ws.numel(), _stream()), "ltsnet_pivot_mds")
    out = (Y, piv, (eig[0], eig[1]))
    return out + (dist,) if return_dist else out


def quality_workspace(n: int, nnz_graph: int):
    """Workspace for the quality-metric calls (device bytes)."""
    return _workspace(lib().ltsnet_quality_workspace_size(int(n), int(nnz_graph)))


def neighbourhood_preservation(row_ptr, col, Y, ws=None, return_counts: bool = False):
    """NP with r = 2 (Sec. 4) over every vertex.  Returns NP, or (NP, b, c)
    with the per-vertex ball sizes b and intersections c (int32 [n] on the
    GPU) if return_counts."""
    torch = _torch()
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    Y = _dev(Y, torch.float32)
    n = row_ptr.numel() - 1
    if ws is None:
        ws = quality_workspace(n, col.numel())
    b = torch.empty((n,), dtype=torch.int32, device="cuda") if return_counts else None
    c = torch.empty((n,), dtype=torch.int32, device="cuda") if return_counts else None
    npv = ctypes.c_double()
    _check(lib().ltsnet_neighbourhood_preservation(_ptr(row_ptr), _ptr(col), n, _ptr(Y), _ptr(b), _ptr(c),
                                                   ctypes.byref(npv), _ptr(ws), ws.numel(), _stream()),
           "ltsnet_neighbourhood_preservation")
    return (npv.value, b, c) if return_counts else npv.value


def stress(row_ptr, col, Y, sources=None, ws=None):
    """ST (Sec. 4) at its optimal scale over the pairs (s, j), s in sources
    (all vertices if None).  Returns (ST, alpha, pairs, skipped pairs)."""
    torch = _torch()
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    Y = _dev(Y, torch.float32)
    n = row_ptr.numel() - 1
    src = torch.arange(n, dtype=torch.int32, device="cuda") if sources is None else _dev(sources, torch.int32)
    if ws is None:
        ws = quality_workspace(n, col.numel())
    out = (ctypes.c_double * 4)()
    _check(lib().ltsnet_stress(_ptr(row_ptr), _ptr(col), n, _ptr(Y), _ptr(src), src.numel(), out, _ptr(ws),
                               ws.numel(), _stream()), "ltsnet_stress")
    return out[0], out[1], int(out[2]), int(out[3])


def calibrate(hop, cnt, perplexity: float, tol: float = 1e-5, max_steps: int = 100):
    """Beta search (Eq. 3).  Returns (beta f64 [n], pcond f64 [n,k],
    converged uint8 [n])."""
    torch = _torch()
    n, k = hop.shape
    beta = torch.empty((n,), dtype=torch.float64, device="cuda")
    pcond = torch.empty((n, k), dtype=torch.float64, device="cuda")
    conv = torch.empty((n,), dtype=torch.uint8, device="cuda")
    _check(lib().ltsnet_calibrate(_ptr(hop), _ptr(cnt), n, k, float(perplexity), float(tol), int(max_steps),
                                  _ptr(beta), _ptr(pcond), _ptr(conv), _stream()), "ltsnet_calibrate")
    return beta, pcond, conv


def symmetrize(nbr, cnt, pcond):
    """Eq. 2.  Returns (P_row int64 [n+1], P_col int32 [nnz], P_val f32 [nnz])."""
    torch = _torch()
    n, k = nbr.shape
    cap = int(lib().ltsnet_symmetrize_max_nnz(n, k))
    P_row = torch.empty((n + 1,), dtype=torch.int64, device="cuda")
    P_col = torch.empty((max(cap, 1),), dtype=torch.int32, device="cuda")
    P_val = torch.empty((max(cap, 1),), dtype=torch.float32, device="cuda")
    ws = _workspace(lib().ltsnet_symmetrize_workspace_size(n, k))
    nnz = ctypes.c_int64(0)
    _check(lib().ltsnet_symmetrize(_ptr(nbr), _ptr(cnt), _ptr(pcond), n, k, _ptr(P_row), _ptr(P_col), _ptr(P_val),
                                   cap, ctypes.byref(nnz), _ptr(ws), ws.numel(), _stream()), "ltsnet_symmetrize")
    m = nnz.value
    return P_row, P_col[:m].clone(), P_val[:m].clone()


def symmetrize_static(nbr, cnt, pcond):
    """Same as symmetrize() but with the library's built-in scratch array
    instead of a workspace (for callers that cannot allocate device memory
    at that point; limit 2 n k <= 2^18).  The outputs are still the caller's."""
    torch = _torch()
    n, k = nbr.shape
    cap = int(lib().ltsnet_symmetrize_max_nnz(n, k))
    P_row = torch.empty((n + 1,), dtype=torch.int64, device="cuda")
    P_col = torch.empty((max(cap, 1),), dtype=torch.int32, device="cuda")
    P_val = torch.empty((max(cap, 1),), dtype=torch.float32, device="cuda")
    nnz = ctypes.c_int64(0)
    _check(lib().ltsnet_symmetrize_static(_ptr(nbr), _ptr(cnt), _ptr(pcond), n, k, _ptr(P_row), _ptr(P_col),
                                          _ptr(P_val), cap, ctypes.byref(nnz), _stream()), "ltsnet_symmetrize_static")
    m = nnz.value
    return P_row, P_col[:m].clone(), P_val[:m].clone()


def bfs_order(row_ptr, col):
    """Breadth-first renumbering.  Returns (order, inv, reordered): order[new]
    = old, inv[old] = new (int32 CUDA tensors)."""
    torch = _torch()
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    n = row_ptr.numel() - 1
    order = torch.empty((n,), dtype=torch.int32, device="cuda")
    inv = torch.empty((n,), dtype=torch.int32, device="cuda")
    ws = _workspace(lib().ltsnet_bfs_order_workspace_size(n))
    r = ctypes.c_int32(0)
    _check(lib().ltsnet_bfs_order(_ptr(row_ptr), _ptr(col), n, _ptr(order), _ptr(inv), ctypes.byref(r), _ptr(ws),
                                  ws.numel(), _stream()), "ltsnet_bfs_order")
    return order, inv, bool(r.value)


def affinities(row_ptr, col, perplexity: float, tol: float = 1e-5, max_steps: int = 100):
    """C0 of Alg. 3 on the GPU: partial BFS, calibration, symmetrisation."""
    k = int(math.ceil(3.0 * perplexity - 1e-9))
    nbr, hop, cnt = knn_bfs(row_ptr, col, k)
    beta, pcond, conv = calibrate(hop, cnt, perplexity, tol, max_steps)
    P = symmetrize(nbr, cnt, pcond)
    return dict(nbr=nbr, hop=hop, cnt=cnt, beta=beta, pcond=pcond, converged=conv, P=P)


def gradient(P, Y, stage: Stage, params: Params | None = None, parts: bool = False, ws=None):
    """One gradient of the tsNET cost at Y.  Returns (grad [n,2] f32,
    parts [n,6] f32 or None, terms [8] f64)."""
    torch = _torch()
    params = params or Params()
    P_row, P_col, P_val = P
    Y = Y.contiguous()
    n = Y.shape[0]
    cp = params.to_c()
    grad = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    pt = torch.empty((n, 6), dtype=torch.float32, device="cuda") if parts else None
    terms = torch.empty((8,), dtype=torch.float64, device="cuda")
    need = lib().ltsnet_gradient_workspace_size(n, ctypes.byref(cp))
    if need == 0:
        raise LtsnetError(-1, "ltsnet_gradient_workspace_size")
    if ws is None or ws.numel() < need:
        ws = _workspace(need)
    st = stage.to_c()
    _check(lib().ltsnet_gradient(_ptr(P_row), _ptr(P_col), _ptr(P_val), n, _ptr(Y), ctypes.byref(st),
                                 ctypes.byref(cp), _ptr(grad), _ptr(pt), _ptr(terms), _ptr(ws), ws.numel(),
                                 _stream()), "ltsnet_gradient")
    _check(lib().ltsnet_poll_status(_ptr(ws), ws.numel(), _stream()), "ltsnet_gradient (device)")
    return grad, pt, terms


VARIANTS = {"bh": 1, "fit": 2}


def gradient_quadtree(P, Y, stage: Stage, params: Params | None = None, theta: float = 0.5, variant: str = "bh",
                      parts: bool = False, ws=None):
    """BH-tsNET ("bh", Alg. 1) or FIt-tsNET ("fit", Alg. 2) gradient at Y:
    the repulsion and/or entropy from the quadtree with opening parameter
    theta.  Returns (grad [n,2] f32, parts [n,6] f32 or None, (Z, S))."""
    torch = _torch()
    params = params or Params()
    P_row, P_col, P_val = P
    Y = Y.contiguous()
    n = Y.shape[0]
    cp = params.to_c()
    v = VARIANTS[variant]
    need = lib().ltsnet_gradient_quadtree_workspace_size(n, ctypes.byref(cp), v)
    if need == 0:
        raise LtsnetError(-1, "ltsnet_gradient_quadtree_workspace_size")
    if ws is None or ws.numel() < need:
        ws = _workspace(need)
    grad = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    pt = torch.empty((n, 6), dtype=torch.float32, device="cuda") if parts else None
    terms = (ctypes.c_double * 2)()
    st = stage.to_c()
    _check(lib().ltsnet_gradient_quadtree(_ptr(P_row), _ptr(P_col), _ptr(P_val), n, _ptr(Y), ctypes.byref(st),
                                          ctypes.byref(cp), float(theta), v, _ptr(grad), _ptr(pt), terms, _ptr(ws),
                                          ws.numel(), _stream()), "ltsnet_gradient_quadtree")
    return grad, pt, (terms[0], terms[1])


def optimize_quadtree(P, Y, update, gains, start_iter: int, n_iter: int, params: Params | None = None,
                      theta: float = 0.5, variant: str = "bh", ws=None):
    """n_iter descent steps of BH-tsNET ("bh") or FIt-tsNET ("fit") from
    global iteration start_iter; Y, update and gains are updated in place."""
    params = params or Params()
    P_row, P_col, P_val = P
    n = Y.shape[0]
    cp = params.to_c()
    v = VARIANTS[variant]
    need = lib().ltsnet_optimize_quadtree_workspace_size(n, ctypes.byref(cp), v)
    if need == 0:
        raise LtsnetError(-1, "ltsnet_optimize_quadtree_workspace_size")
    if ws is None or ws.numel() < need:
        ws = _workspace(need)
    _check(lib().ltsnet_optimize_quadtree(_ptr(P_row), _ptr(P_col), _ptr(P_val), n, ctypes.byref(cp), float(theta),
                                          v, _ptr(Y), _ptr(update), _ptr(gains), int(start_iter), int(n_iter),
                                          _ptr(ws), ws.numel(), _stream()), "ltsnet_optimize_quadtree")
    return Y


def cost(P, Y, stage: Stage, params: Params | None = None, grad_pvals: bool = False, ws=None):
    """The cost of Eq. 1 at Y: returns (cost f64[4] tensor = C_KL, C_CMP,
    C_ENT, total; dC/dP_val f32[nnz] tensor or None)."""
    torch = _torch()
    params = params or Params()
    P_row, P_col, P_val = P
    Y = Y.contiguous()
    n = Y.shape[0]
    cp = params.to_c()
    out = torch.empty((4,), dtype=torch.float64, device="cuda")
    dP = torch.empty_like(P_val) if grad_pvals else None
    need = lib().ltsnet_gradient_workspace_size(n, ctypes.byref(cp))
    if need == 0:
        raise LtsnetError(-1, "ltsnet_gradient_workspace_size")
    if ws is None or ws.numel() < need:
        ws = _workspace(need)
    st = stage.to_c()
    _check(lib().ltsnet_cost(_ptr(P_row), _ptr(P_col), _ptr(P_val), n, _ptr(Y), ctypes.byref(st), ctypes.byref(cp),
                             _ptr(out), _ptr(dP), _ptr(ws), ws.numel(), _stream()), "ltsnet_cost")
    _check(lib().ltsnet_poll_status(_ptr(ws), ws.numel(), _stream()), "ltsnet_cost (device)")
    return out, dP


def grad_pvals(P, Y, stage: Stage, params: Params | None = None, ws=None):
    """dC/dP_val (f32 [nnz] tensor) at Y by ltsnet_grad_pvals."""
    torch = _torch()
    params = params or Params()
    P_row, P_col, P_val = P
    Y = Y.contiguous()
    n = Y.shape[0]
    cp = params.to_c()
    dP = torch.empty_like(P_val)
    need = lib().ltsnet_gradient_workspace_size(n, ctypes.byref(cp))
    if need == 0:
        raise LtsnetError(-1, "ltsnet_gradient_workspace_size")
    if ws is None or ws.numel() < need:
        ws = _workspace(need)
    st = stage.to_c()
    _check(lib().ltsnet_grad_pvals(_ptr(P_row), _ptr(P_col), _ptr(P_val), n, _ptr(Y), ctypes.byref(st),
                                   ctypes.byref(cp), _ptr(dP), _ptr(ws), ws.numel(), _stream()), "ltsnet_grad_pvals")
    _check(lib().ltsnet_poll_status(_ptr(ws), ws.numel(), _stream()), "ltsnet_grad_pvals (device)")
    return dP


def _cost_function():
    torch = _torch()

    class LTsNetCost(torch.autograd.Function):
        """C(Y, P_val) of Eq. 1 as a differentiable scalar (f64, 0-dim):
        forward by ltsnet_cost, backward by ltsnet_gradient (dC/dY, the
        interpolated gradient of Eq. 6 and Eq. 8) and ltsnet_grad_pvals
        (dC/dP_val).  P_row and P_col are structure, not differentiated.

        The cost of Eq. 1 has no exaggeration factor (early exaggeration
        scales P in the optimiser's gradient only), so a stage with
        exaggeration != 1 is rejected rather than given a backward that is not
        the derivative of the forward.

        recompute=False keeps dC/dY (8n bytes) and dC/dP_val (4 nnz bytes)
        from the forward pass until backward; recompute=True keeps only
        references to the inputs and recomputes the grid fields, the gradient
        and dC/dP_val (only if P_val needs a gradient) in backward, so that
        nothing of size nnz is held between the two passes."""

        @staticmethod
        def forward(ctx, Y, P_val, P_row, P_col, stage, params, recompute=False):
            if stage.exaggeration != 1.0:
                raise ValueError("LTsNetCost: the cost of Eq. 1 has no exaggeration; use a stage with "
                                 "exaggeration = 1")
            P = (P_row, P_col, P_val.detach().contiguous())
            Yd = Y.detach().contiguous()
            ctx.stage, ctx.params, ctx.recompute = stage, params, bool(recompute)
            if recompute:
                c, _ = cost(P, Yd, stage, params, grad_pvals=False)
                ctx.save_for_backward(Yd, P[2], P_row, P_col)
            else:
                c, dP = cost(P, Yd, stage, params, grad_pvals=True)
                g, _, _ = gradient(P, Yd, stage, params)
                ctx.save_for_backward(g, dP)
            return c[3].clone()

        @staticmethod
        def backward(ctx, go):
            if ctx.recompute:
                Yd, Pv, P_row, P_col = ctx.saved_tensors
                P = (P_row, P_col, Pv)
                g = gradient(P, Yd, ctx.stage, ctx.params)[0] if ctx.needs_input_grad[0] else None
                dP = grad_pvals(P, Yd, ctx.stage, ctx.params) if ctx.needs_input_grad[1] else None
            else:
                g, dP = ctx.saved_tensors
            s = go.to(torch.float32)
            return (g * s if g is not None else None, dP * s if dP is not None else None,
                    None, None, None, None, None)

    return LTsNetCost


_LTsNetCost = None


def ltsnet_cost_fn():
    """The torch.autograd.Function LTsNetCost: apply(Y, P_val, P_row, P_col,
    stage, params, recompute=False) -> cost."""
    global _LTsNetCost
    if _LTsNetCost is None:
        _LTsNetCost = _cost_function()
    return _LTsNetCost


def optimize(P, Y, update, gains, start_iter: int, n_iter: int, params: Params | None = None, ws=None,
             sync: bool = True):
    """Runs iterations [start_iter, start_iter+n_iter) of the schedule in
    place on (Y, update, gains)."""
    params = params or Params()
    P_row, P_col, P_val = P
    n = Y.shape[0]
    cp = params.to_c()
    need = lib().ltsnet_optimize_workspace_size(n, ctypes.byref(cp))
    if need == 0:
        raise LtsnetError(-1, "ltsnet_optimize_workspace_size")
    if ws is None or ws.numel() < need:
        ws = _workspace(need)
    _check(lib().ltsnet_optimize(_ptr(P_row), _ptr(P_col), _ptr(P_val), n, ctypes.byref(cp), _ptr(Y), _ptr(update),
                                 _ptr(gains), int(start_iter), int(n_iter), _ptr(ws), ws.numel(), _stream()),
           "ltsnet_optimize")
    if sync:
        _check(lib().ltsnet_poll_status(_ptr(ws), ws.numel(), _stream()), "ltsnet_optimize (device)")
    return ws


def run_workspace(n: int, nnz_graph: int, params: Params):
    cp = params.to_c()
    need = lib().ltsnet_run_workspace_size(n, nnz_graph, ctypes.byref(cp))
    if need == 0:
        raise LtsnetError(-1, "ltsnet_run_workspace_size")
    return _workspace(need)


def run(row_ptr, col, Y0, params: Params | None = None, ws=None):
    """Alg. 3 (without Pivot-MDS): C0 then the whole schedule.  Y0 is a
    [n,2] float32 CUDA tensor; returns the final layout (a new tensor)."""
    torch = _torch()
    params = params or Params()
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    Y = Y0.to(device="cuda", dtype=torch.float32).contiguous().clone()
    n = Y.shape[0]
    cp = params.to_c()
    if ws is None:
        ws = run_workspace(n, col.numel(), params)
    rc = lib().ltsnet_run(_ptr(row_ptr), _ptr(col), n, ctypes.byref(cp), _ptr(Y), _ptr(ws), ws.numel(), _stream())
    _check(rc, "ltsnet_run")
    return Y, rc


def _batch_arrays(graphs, Y0s):
    import numpy as np
    torch = _torch()
    ns = [int(g.row_ptr.shape[0] - 1) for g in graphs]
    ms = [int(g.col.shape[0]) for g in graphs]
    vtx_off = np.zeros(len(graphs) + 1, np.int64)
    edge_off = np.zeros(len(graphs) + 1, np.int64)
    vtx_off[1:] = np.cumsum(ns)
    edge_off[1:] = np.cumsum(ms)
    rp = torch.from_numpy(np.concatenate([np.asarray(g.row_ptr, np.int64) for g in graphs])).cuda()
    col = torch.from_numpy(np.concatenate([np.asarray(g.col, np.int32) for g in graphs])).cuda()
    Y = torch.from_numpy(np.concatenate([np.asarray(y, np.float32) for y in Y0s])).cuda().contiguous()
    return vtx_off, edge_off, rp, col, Y


def run_batched(graphs, Y0s, params: Params | None = None, workers: int = 16, mode: int = BATCH_ONE_LAUNCH,
                fft_blocks: int = 0, spread_blocks: int = 0, return_boxes: bool = False, max_boxes=None):
    """The method on many independent graphs at once (ltsnet_run_batched).
    graphs: objects with row_ptr (int64 [n+1]) and col (int32) numpy arrays;
    Y0s: matching float32 [n,2] arrays.  mode BATCH_ONE_LAUNCH runs the loop
    with one launch per phase over all graphs (fft_blocks / spread_blocks
    blocks per graph, 0 = the library's defaults), BATCH_PER_GRAPH one
    ltsnet_run per graph on `workers` host threads.  max_boxes: optional
    per-graph grid caps (0 = params.max_boxes).  Returns (Y, vtx_off) --
    all final layouts in one [sum n, 2] CUDA tensor, graph g in rows
    vtx_off[g]:vtx_off[g+1] -- and, if return_boxes, the largest box count
    per dimension of each graph's grid."""
    import numpy as np
    params = params or Params()
    vtx_off, edge_off, rp, col, Y = _batch_arrays(graphs, Y0s)
    cp = params.to_c()
    boxes = np.zeros(len(graphs), np.int32)
    caps = None
    if max_boxes is not None:
        caps = np.ascontiguousarray(np.asarray(max_boxes, dtype=np.int32))
        if caps.shape != (len(graphs),):
            raise ValueError("max_boxes: one cap per graph")
    cfg = CBatchConfig(int(mode), max(1, min(int(workers), 64)), int(fft_blocks), int(spread_blocks),
                       boxes.ctypes.data, caps.ctypes.data if caps is not None else None)
    need = lib().ltsnet_run_batched_workspace_size(len(graphs), vtx_off.ctypes.data, edge_off.ctypes.data,
                                                    ctypes.byref(cp), ctypes.byref(cfg))
    if need == 0:
        raise LtsnetError(-1, "ltsnet_run_batched_workspace_size")
    ws = _workspace(need)
    rc = lib().ltsnet_run_batched(len(graphs), vtx_off.ctypes.data, edge_off.ctypes.data, _ptr(rp), _ptr(col),
                                  ctypes.byref(cp), _ptr(Y), _ptr(ws), ws.numel(), ctypes.byref(cfg), _stream())
    _check(rc, "ltsnet_run_batched")
    return (Y, vtx_off, boxes) if return_boxes else (Y, vtx_off)


def _tune_key(graphs, params: Params, max_boxes=None) -> str:
    """Cache key of a batch: buckets of its median and largest graph size
    (powers of 2), of its largest grid (nodes per side at the largest cap) and
    of its mean entries per row of the graph (powers of 2)."""
    import numpy as np
    ns = np.array([int(g.row_ptr.shape[0] - 1) for g in graphs])
    deg = float(np.mean([g.col.shape[0] / max(1, g.row_ptr.shape[0] - 1) for g in graphs]))
    cap = params.max_boxes
    if max_boxes is not None:
        caps = np.asarray(max_boxes)
        cap = int(np.where(caps > 0, caps, params.max_boxes).max())
    b = lambda x: int(np.ceil(np.log2(max(1.0, x))))  # noqa: E731
    return (f"n{b(np.median(ns))}-{b(ns.max())}_M{params.nodes_per_box * cap}_d{b(deg)}"
            f"_p{params.perplexity:g}")


def autotune_batched(graphs, Y0s, params: Params | None = None, cache: str | None = None, iters: int = 40,
                     candidates=((2, 4), (4, 8), (8, 8), (8, 16), (16, 16)), workers: int = 16, max_boxes=None):
    """Picks the launch shape (FFT blocks, spread blocks per graph) of the
    one-launch batched form by timing each candidate on the batch itself
    (`iters` iterations of the default schedule's second stage, per-graph grid
    caps `max_boxes` as in run_batched) and keeps the fastest in a JSON cache
    keyed by _tune_key.  Returns (fft_blocks, spread_blocks, timings)."""
    import json
    import os
    import time
    torch = _torch()
    params = params or Params()
    key = _tune_key(graphs, params, max_boxes)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            return tuple(table[key]["best"]) + (table[key]["ms"],)
    probe = Params(**{**params.__dict__, "stages": [Stage(iters, 1.0, 0.01, 0.6, 1.0, 0.8)]})
    ms = {}
    for fb, sb in candidates:
        run_batched(graphs, Y0s, probe, workers=workers, fft_blocks=fb, spread_blocks=sb,
                    max_boxes=max_boxes)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_batched(graphs, Y0s, probe, workers=workers, fft_blocks=fb, spread_blocks=sb, max_boxes=max_boxes)
        torch.cuda.synchronize()
        ms[f"{fb},{sb}"] = round((time.perf_counter() - t0) * 1e3, 2)
    best = min(ms, key=ms.get)
    fb, sb = (int(x) for x in best.split(","))
    if cache:
        table[key] = {"best": [fb, sb], "ms": ms}
        with open(cache, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return fb, sb, ms


def run_host(row_ptr, col, Y, params: Params | None = None, ws=None):
    """Same as run() with HOST numpy arrays (the library copies them in and the
    layout back); Y (float32 [n,2], C-contiguous) is updated in place."""
    import numpy as np
    params = params or Params()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    assert Y.dtype == np.float32 and Y.flags["C_CONTIGUOUS"]
    n = Y.shape[0]
    cp = params.to_c()
    if ws is None:
        ws = run_workspace(n, col.size, params)
    rc = lib().ltsnet_run_host(row_ptr.ctypes.data_as(ctypes.c_void_p), col.ctypes.data_as(ctypes.c_void_p), n,
                               ctypes.byref(cp), Y.ctypes.data_as(ctypes.c_void_p), _ptr(ws), ws.numel(), _stream())
    _check(rc, "ltsnet_run_host")
    return Y, rc


def launch_count() -> int:
    return int(lib().ltsnet_launch_count())


def profile_begin(kernel: int, max_launches: int):
    _check(lib().ltsnet_profile_begin(kernel, max_launches), "ltsnet_profile_begin")


def profile_end(kernel: int):
    ms = ctypes.c_double(0)
    cnt = ctypes.c_int32(0)
    _check(lib().ltsnet_profile_end(kernel, ctypes.byref(ms), ctypes.byref(cnt)), "ltsnet_profile_end")
    return ms.value, cnt.value
