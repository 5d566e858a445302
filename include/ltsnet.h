/*
 * ltsnet.h -- C ABI of the GB300 L-tsNET library (libltsnet.so).
 *
 * L-tsNET (Meidiana, Hong, Ma, "BH-tsNET, FIt-tsNET, L-tsNET: Fast tsNET
 * Algorithms for Large Graph Drawing", arXiv 2509.19785) lays out a graph by
 * minimising the tsNET cost (Eq. 1) of a 2-D layout Y.  Alg. 3 takes a graph,
 * a perplexity u, a number of intervals I and a number of interpolation points
 * P and returns the layout; the calls below follow that statement.
 *
 * Conventions shared by every call:
 *  - Pointers are DEVICE pointers unless the comment says "host".
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream) and is asynchronous unless the comment says "synchronous".
 *  - The library never allocates or frees device memory.  The caller owns
 *    every buffer, including the workspace `ws` (`ws_bytes` long, 256-byte
 *    aligned), whose size the matching *_workspace_size call returns.
 *  - Every call returns an ltsnet_status.  Argument errors are detected on the
 *    host and returned before anything is enqueued.  Errors found by a kernel
 *    (a vertex id out of range, a non-finite coordinate, a loop that hit its
 *    iteration cap) are recorded in a status word inside the workspace; the
 *    synchronous calls return it, and ltsnet_poll_status reads it for the
 *    asynchronous ones.  No kernel traps.
 *  - Layout Y is row-major float[n][2] (x_i, y_i); gradients use the same
 *    layout.  Graphs are CSR with int64 row offsets and int32 column ids, both
 *    directions of every undirected edge stored; self-loops and duplicate
 *    entries are allowed and ignored.
 */
#ifndef LTSNET_H
#define LTSNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ltsnet_stream; /* = cudaStream_t */

typedef enum {
    LTSNET_OK = 0,
    LTSNET_WARN_NOT_CONVERGED = 1, /* some rows missed the perplexity target (the "perplexity too low" case of Sec. 4.1) */
    LTSNET_ERR_INVALID_ARG = -1,
    LTSNET_ERR_WORKSPACE = -2,     /* workspace or output capacity too small */
    LTSNET_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    LTSNET_ERR_DEVICE_TIMEOUT = -4,/* a device loop reached its iteration cap */
    LTSNET_ERR_NONFINITE = -5,     /* NaN/Inf in the layout or the gradient */
    LTSNET_ERR_BAD_GRAPH = -6      /* a column id outside [0, n) */
} ltsnet_status;

/* One descent stage.  Sec. 2.1: the multipliers lambda_KL, lambda_c, lambda_r
 * of the three cost terms (Eq. 1) change between stages; the paper gives no
 * values.  `exaggeration` multiplies P in the attractive term (1 = none);
 * `momentum` is the optimiser's momentum for the stage. */
typedef struct {
    int32_t iters;
    float lambda_kl;
    float lambda_c;
    float lambda_r;
    float exaggeration;
    float momentum;
} ltsnet_stage;

/* Method parameters.  ltsnet_default_params() fills every field. */
typedef struct {
    float perplexity;      /* u of Eq. 3; k = ceil(3u) neighbours per vertex (Sec. 3.1) */
    float eps;             /* entropy kernel regulariser, 1/20 (Sec. 3.3) */
    int32_t nodes_per_box; /* P of Alg. 3, interpolation nodes per interval: 2, 3, 4 or 5 (default 3) */
    float box_width_max;   /* grid rule: I = max(min_boxes, ceil(extent / box_width_max)) ... */
    int32_t min_boxes;     /* ... rounded up to a 5-smooth size ... */
    int32_t max_boxes;     /* ... and capped here (the cap widens the boxes); default 640;
                              2 * nodes_per_box * max_boxes (the FFT length) <= 4096 */
    float learning_rate;   /* <= 0: max(200, n/12) */
    int32_t beta_max_steps;/* beta search cap (default 100) */
    double beta_tol;       /* |H_i - ln u| tolerance (default 1e-5) */
    int32_t n_stages;      /* stage schedule; stages is a HOST pointer */
    const ltsnet_stage* stages;
    int32_t flags;         /* LTSNET_FLAG_* */
    int32_t conv_mode;     /* grid convolution (Sec. 2.3): LTSNET_CONV_* */
} ltsnet_params;

/* conv_mode: how the kernels are convolved with the charge grids (the
 * interpolation of Sec. 2.3 and Sec. 3.3; the paper uses FFTs).
 * LTSNET_CONV_FFT: FP32 FFTs of the zero-padded grids (default).
 * LTSNET_CONV_DFT_GEMM: the same sums as real DFT matrix products on the
 * tensor cores (tcgen05), every FP32 operand split into three BF16 terms
 * (v = v0 + v1 + v2) and each product taken as the six term products
 * a_i b_j with i + j <= 2, accumulated in FP32; not with LTSNET_FLAG_PLAIN.
 * Its workspace adds about 400 (nodes_per_box max_boxes)^2 bytes (1.45 GB at
 * P = 3 and 640 boxes). */
#define LTSNET_CONV_FFT 0
#define LTSNET_CONV_DFT_GEMM 1

/* flags: LTSNET_FLAG_PLAIN selects the unfused FP32 baseline form of the loop
 * (atomic spread in input order, separate gather/attraction/update kernels)
 * instead of the optimised form (box-sorted deterministic spread, fused
 * gather + attraction + compression + update). */
#define LTSNET_FLAG_PLAIN 1
/* flags: LTSNET_FLAG_NO_REORDER keeps the input's vertex numbering inside
 * ltsnet_run / ltsnet_run_host.  By default those calls renumber the vertices
 * in breadth-first order (Cuthill-McKee) after the partial BFS, so that the
 * attraction pass reads neighbour coordinates from nearby memory; the result
 * is returned in the input's numbering and differs only in floating-point
 * summation order.  Graphs with more than 4096 BFS levels are not renumbered. */
#define LTSNET_FLAG_NO_REORDER 2

/* Largest supported k (partial BFS neighbours per vertex). */
#define LTSNET_MAX_K 4096

/* Defaults: perplexity 30, eps 1/20 (Sec. 3.3), P = 3, box_width_max 0.25,
 * min_boxes 50, max_boxes 640, automatic learning rate, beta search 100 steps
 * / 1e-5, the two-stage schedule of ltsnet_default_stages (1000 iterations).
 * Only eps comes from the paper; the rest are this library's readings
 * (no counterpart in the paper).  The grid defaults hold the interpolated
 * repulsion and entropy sums and Z within 5e-3 relative L2 of the exact
 * O(n^2) sums on the layouts of whole runs (the entropy kernel
 * 1/(eps + d^2) is only sqrt(eps) = 0.22 wide: boxes of width 0.5 leave its
 * sums 1.7e-2 off on clustered layouts), as long as max_boxes does not bind
 * (layout extent <= 160). */
ltsnet_params ltsnet_default_params(void);

/* Writes the default schedule for `total_iters` iterations into `out` (host,
 * room for 2) and returns the number of stages: 250 iterations of
 * (lambda_KL, lambda_c, lambda_r) = (1, 1.2, 0) with momentum 0.5, then the
 * rest with (1, 0.01, 0.6) and momentum 0.8.  Sec. 2.1 says the multipliers
 * change between stages but gives no values: these are a reading (no
 * counterpart in the paper). */
int32_t ltsnet_default_stages(int32_t total_iters, ltsnet_stage* out);

/* Host: a static description of a status code (no counterpart in the paper;
 * the status calls below are error plumbing). */
const char* ltsnet_status_string(ltsnet_status s);

/* Host: text of the last CUDA runtime failure seen by this library on the
 * calling thread (name, description and source location), "" if none.  The
 * string is owned by the library and valid until the thread's next failure.
 * No counterpart in the paper. */
const char* ltsnet_last_cuda_error(void);

/* Synchronous: waits for `stream`, returns the status word recorded in `ws`
 * by earlier asynchronous calls and clears it.  No counterpart in the paper. */
ltsnet_status ltsnet_poll_status(void* ws, size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * C0 step 1 -- partial BFS k-nearest neighbours (Sec. 3.1, "partial BFS";
 * Alg. 3 preprocessing loop).  For every source s: breadth-first search in
 * FIFO order over the adjacency lists in their stored order, a vertex counting
 * as visited when first reached, stopping as soon as k vertices other than s
 * are visited.  The paper breaks ties randomly; this library breaks them by
 * that deterministic discovery order, so the output is a function of the CSR.
 *   row_ptr int64[n+1], col int32[row_ptr[n]]       graph (device)
 *   nbr  int32[n][k]   neighbours of s in discovery order, -1 padded
 *   hop  uint16[n][k]  their hop distances (non-decreasing along a row), 0 pad
 *   cnt  int32[n]      neighbours found, = min(k, |component(s)| - 1)
 * 1 <= k <= LTSNET_MAX_K.  A column id outside [0, n) is skipped and recorded
 * as LTSNET_ERR_BAD_GRAPH in the workspace status word.  ws >= 256 bytes.
 * ------------------------------------------------------------------------- */
ltsnet_status ltsnet_knn_bfs(const int64_t* row_ptr, const int32_t* col, int32_t n, int32_t k,
                             int32_t* nbr, uint16_t* hop, int32_t* cnt,
                             void* ws, size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * C0 step 2 -- perplexity calibration (Eq. 3 and the definition of the
 * perplexity u beneath it).  Per row i, with d_ij the hop distance:
 *   p_{j|i} = exp(-beta_i d_ij^2) / sum_l exp(-beta_i d_il^2),
 *   beta_i = 1/(2 sigma_i^2) chosen so that -sum_j p_{j|i} ln p_{j|i} = ln u.
 * Search in FP64: beta = 1; raise it (double, or bisect once bracketed) while
 * the entropy is above ln u, lower it (halve, or bisect) while below; stop at
 * |H - ln u| < tol or after max_steps evaluations; p is evaluated at the final
 * beta.
 *   beta       f64[n]        converged u8[n] (1 iff the tolerance was met)
 *   pcond      f64[n][k]     p_{j|i} aligned with nbr/hop, 0 beyond cnt
 * Rows with no neighbours get beta = 1, converged = 0.
 * ------------------------------------------------------------------------- */
ltsnet_status ltsnet_calibrate(const uint16_t* hop, const int32_t* cnt, int32_t n, int32_t k,
                               double perplexity, double tol, int32_t max_steps,
                               double* beta, double* pcond, uint8_t* converged,
                               ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * C0 step 3 -- symmetrisation (Eq. 2): p_ij = (p_{j|i} + p_{i|j}) / (2n) over
 * the union of the supports of the conditional rows, as CSR with every row's
 * columns ascending.  The sum and the division are done in FP64 and rounded
 * once to FP32.  Synchronous (returns nnz on the host).
 *   P_row int64[n+1], P_col int32[cap], P_val f32[cap]; cap >= nnz, and
 *   nnz <= ltsnet_symmetrize_max_nnz(n, k).  *nnz_out (host) gets nnz.
 * Returns LTSNET_ERR_WORKSPACE if cap < nnz (P_row is still complete).
 * ------------------------------------------------------------------------- */
int64_t ltsnet_symmetrize_max_nnz(int32_t n, int32_t k);
size_t ltsnet_symmetrize_workspace_size(int32_t n, int32_t k);
ltsnet_status ltsnet_symmetrize(const int32_t* nbr, const int32_t* cnt, const double* pcond,
                                int32_t n, int32_t k,
                                int64_t* P_row, int32_t* P_col, float* P_val, int64_t cap,
                                int64_t* nnz_out, void* ws, size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * ltsnet_symmetrize without a workspace argument (no counterpart in the
 * paper; an interface for callers that cannot allocate device memory where
 * they need this step: plug-ins and embedded hosts handed a fixed
 * device-memory budget that forbid allocation, and loops that must not pay
 * for cudaMalloc's implicit synchronisation).  The scratch is a device array
 * built into the library (about 5.2 MB on every GPU that loads it, held until
 * the process exits); nothing is allocated by the call.  Limit:
 * 2 * n * k <= ltsnet_symmetrize_static_max_entries() (2^18); larger inputs
 * return LTSNET_ERR_WORKSPACE without touching the GPU.  The first call on a
 * device looks up the array's device address there (cudaGetSymbolAddress),
 * so make that first call before any stream capture.  All calls share the
 * array: calls whose GPU work overlaps (other streams or threads) race.
 * Synchronous, same arguments and results as ltsnet_symmetrize.
 * ------------------------------------------------------------------------- */
int64_t ltsnet_symmetrize_static_max_entries(void);
ltsnet_status ltsnet_symmetrize_static(const int32_t* nbr, const int32_t* cnt, const double* pcond,
                                       int32_t n, int32_t k,
                                       int64_t* P_row, int32_t* P_col, float* P_val, int64_t cap,
                                       int64_t* nnz_out, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * Breadth-first vertex renumbering (a memory-locality aid; no counterpart in
 * the paper).  order[new] = old in the discovery order of a FIFO BFS that
 * scans adjacency lists in stored order, starting at vertex 0 and restarting
 * at the smallest unvisited vertex for each further component; inv is the
 * inverse.  *reordered (host) = 0 and order/inv untouched if the graph has
 * more than 4096 BFS levels.  Synchronous.  ltsnet_run applies it internally
 * unless LTSNET_FLAG_NO_REORDER is set; callers of ltsnet_optimize can apply
 * it to their own P (relabel rows and columns) for the same effect.
 * ------------------------------------------------------------------------- */
size_t ltsnet_bfs_order_workspace_size(int32_t n);
ltsnet_status ltsnet_bfs_order(const int64_t* row_ptr, const int32_t* col, int32_t n,
                               int32_t* order, int32_t* inv, int32_t* reordered,
                               void* ws, size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * One gradient of the tsNET cost at Y (Alg. 3 loop body without the move):
 *   dC/dX_i = 4 lambda_KL (alpha A_i - (S/Z) R_i) + (lambda_c/n) X_i
 *             - (lambda_r/n^2) E_i
 *   A_i = sum_{j in row i} p_ij (X_i - X_j)/(1 + d_ij^2)   sparse, exact (Eq. 6)
 *   R_i = sum_j (X_i - X_j)/(1 + d_ij^2)^2                  interpolated (Sec. 2.3)
 *   E_i = sum_j (X_i - X_j)/(eps + d_ij^2) = X_i h1 - (h2,h3) interpolated (Eq. 8)
 *   Z   = sum_{i != j} 1/(1 + d_ij^2)                       from the grid, FP64
 *   S   = sum of P_val (1 for a normalised P), alpha = stage exaggeration.
 * The interpolation: lo/hi = min/max over all coordinates, I boxes per
 * dimension by the grid rule of ltsnet_params, nodes_per_box Lagrange nodes
 * per box.  The paper's sums carry the charges (1, x, y, x^2+y^2); this
 * library computes the same sums rearranged exactly: every point spreads its
 * node-local moments S0 = L, S1 = L e, S2 = L |e|^2 (L its Lagrange weight at
 * a node, e its offset from that node in node spacings), which are convolved
 * on the node grid with the kernels (1+d^2)^-2 and 1/(eps+d^2) and with
 * those kernels times the node offset (zero-padded FFT), and gathered back;
 * no FP32 value carries the layout's absolute coordinates.
 *   grad  f32[n][2]       (device)
 *   parts f32[n][6] or NULL: (A_i, R_i, E_i) unscaled, for per-term checks
 *   terms f64[8] or NULL: Z, S, I, h, lo, centre, M, 0
 * ------------------------------------------------------------------------- */
size_t ltsnet_gradient_workspace_size(int32_t n, const ltsnet_params* p);
ltsnet_status ltsnet_gradient(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                              int32_t n, const float* Y, const ltsnet_stage* stage,
                              const ltsnet_params* p, float* grad, float* parts, double* terms,
                              void* ws, size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * The cost of Eq. 1 at Y (entropy term in the reading whose gradient is the
 * Sec. 3.3 kernel) and its derivative with respect to the stored P values:
 *   C_KL  = lambda_KL [sum p ln p + sum p ln(1 + d^2) + S ln Z]   (Eq. 1, Eq. 4)
 *   C_CMP = lambda_c / (2n) sum_i |X_i|^2                          (Eq. 1)
 *   C_ENT = -lambda_r / (4 n^2) sum_{i != j} ln(eps + d_ij^2)      (Eq. 1, reading)
 *   dC/dp_e = lambda_KL (ln p_e + 1 + ln(1 + d_e^2) + ln Z)        (each entry a leaf)
 * The sparse sums are exact; Z and the entropy double sum come from the same
 * grid as ltsnet_gradient (the entropy sum interpolates ln(eps + d^2) in both
 * arguments: sum_t W0[t] (K_ln * W0)[t] - n ln eps, W0 the spread of charge
 * 1).  The exaggeration factor does not enter.  Uses the gradient's workspace
 * (ltsnet_gradient_workspace_size).
 *   cost     f64[4] (device) or NULL: C_KL, C_CMP, C_ENT, total
 *   dC_dPval f32[nnz] (device) or NULL (not both NULL)
 * Column indices outside [0, n) are reported as LTSNET_ERR_BAD_GRAPH.
 * ------------------------------------------------------------------------- */
ltsnet_status ltsnet_cost(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                          int32_t n, const float* Y, const ltsnet_stage* stage,
                          const ltsnet_params* p, double* cost, float* dC_dPval,
                          void* ws, size_t ws_bytes, ltsnet_stream stream);
/* ltsnet_cost with cost = NULL: dC/dp_e only (the derivative of Eq. 1 with
 * respect to each stored entry of P, as above). */
ltsnet_status ltsnet_grad_pvals(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                                int32_t n, const float* Y, const ltsnet_stage* stage,
                                const ltsnet_params* p, float* dC_dPval,
                                void* ws, size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * The descent loop (Alg. 3, "for iterations": gradient, then move every
 * vertex).  Runs iterations [start_iter, start_iter + n_iter) of the stage
 * schedule in `p`, updating Y, update (the previous step) and gains in place:
 *   gain <- gain + 0.2 where sign(g) != sign(update), else gain * 0.8;
 *   gain >= 0.01; update <- momentum*update - lr*gain*g; Y <- Y + update.
 * (The paper does not name its optimiser; this is the t-SNE optimiser of van
 * der Maaten and Hinton, which its C++ code base derives from.)  Start with
 * update = 0, gains = 1.  Resuming from start_iter > 0 with the saved
 * (Y, update, gains) gives the same result as an uninterrupted run.
 * ------------------------------------------------------------------------- */
size_t ltsnet_optimize_workspace_size(int32_t n, const ltsnet_params* p);
ltsnet_status ltsnet_optimize(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                              int32_t n, const ltsnet_params* p, float* Y, float* update,
                              float* gains, int32_t start_iter, int32_t n_iter,
                              void* ws, size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * Whole method (Alg. 3 without the Pivot-MDS initialisation): C0 on the graph,
 * then every iteration of the schedule.  Y holds the initial layout on entry
 * and the final layout on return.  Synchronous; returns the first error, or
 * LTSNET_WARN_NOT_CONVERGED if some rows missed the perplexity target.
 * ltsnet_run_host takes HOST pointers for the graph and Y and does the
 * host<->device copies itself (through the workspace).
 * ------------------------------------------------------------------------- */
size_t ltsnet_run_workspace_size(int32_t n, int64_t nnz_graph, const ltsnet_params* p);
ltsnet_status ltsnet_run(const int64_t* row_ptr, const int32_t* col, int32_t n,
                         const ltsnet_params* p, float* Y, void* ws, size_t ws_bytes,
                         ltsnet_stream stream);
ltsnet_status ltsnet_run_host(const int64_t* row_ptr_host, const int32_t* col_host, int32_t n,
                              const ltsnet_params* p, float* Y_host, void* ws, size_t ws_bytes,
                              ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * Many independent graphs (the batched form of the method): ltsnet_run
 * (Alg. 3) on each of n_graphs graphs, with the same parameters, in one call.
 * The batching has no counterpart in the paper.
 *   vtx_off  int64[n_graphs+1] (HOST): graph g owns vertices
 *            [vtx_off[g], vtx_off[g+1]) of Y (f32 [sum n][2], device, in: Y0,
 *            out: final layouts); vtx_off[0] = 0, every graph non-empty
 *   edge_off int64[n_graphs+1] (HOST): graph g's columns are
 *            col[edge_off[g] .. edge_off[g+1]) (int32, device, local ids)
 *   row_ptr  int64 (device): graph g's n_g+1 local row pointers (from 0) start
 *            at row_ptr[vtx_off[g] + g]
 * Modes (cfg->mode):
 *  LTSNET_BATCH_ONE_LAUNCH: C0 of every graph on cfg->n_workers host threads,
 *    then the whole descent loop with one launch per phase covering every
 *    graph (grid.y = graph; cfg->fft_blocks and cfg->spread_blocks blocks per
 *    graph for the FFT passes and the spread, 0 = 4 and 8), replayed from CUDA
 *    graphs; FFT convolution and the optimised form only (LTSNET_FLAG_PLAIN
 *    and conv_mode 1 return LTSNET_ERR_INVALID_ARG).  Each graph's result
 *    equals ltsnet_run's for that graph alone (every reduction is split the
 *    same way whatever the launch shape).
 *  LTSNET_BATCH_PER_GRAPH: ltsnet_run per graph on cfg->n_workers host
 *    threads, each with its own stream (largest graphs first).
 * cfg->max_boxes (HOST int32[n_graphs], may be NULL): graph g runs with the
 * grid cap max_boxes[g] in place of p->max_boxes where that entry is
 * positive (the same bounds as p->max_boxes apply; an out-of-range cap
 * returns LTSNET_ERR_INVALID_ARG), so a batch can give its large graphs
 * large grids without sizing every graph's grid arrays for them.
 * cfg->max_boxes_used (HOST int32[n_graphs], may be NULL): the largest number
 * of boxes per dimension each graph's grid had during the run (-1 in the
 * per-graph mode): equal to the graph's cap where that cap bound.  Synchronous
 * (waits for `stream` first); returns the first error, else
 * LTSNET_WARN_NOT_CONVERGED if any graph had rows that missed the perplexity
 * target, else LTSNET_OK.
 * ------------------------------------------------------------------------- */
#define LTSNET_BATCH_ONE_LAUNCH 0
#define LTSNET_BATCH_PER_GRAPH 1
typedef struct {
    int32_t mode;            /* LTSNET_BATCH_* */
    int32_t n_workers;       /* host threads, 1..64 */
    int32_t fft_blocks;      /* blocks per graph of the FFT passes, 0..64 (0: 4) */
    int32_t spread_blocks;   /* blocks per graph of the box spread, 0..64 (0: 8) */
    int32_t* max_boxes_used; /* HOST int32[n_graphs] or NULL */
    const int32_t* max_boxes; /* HOST int32[n_graphs] or NULL: per-graph cap of
                                 the boxes per dimension (an entry of 0 takes
                                 p->max_boxes); each graph's grid arrays are
                                 sized for its own cap */
} ltsnet_batch_config;
/* The batched calls (Alg. 3 on every graph; the batching itself has no
 * counterpart in the paper), as described above. */
size_t ltsnet_run_batched_workspace_size(int32_t n_graphs, const int64_t* vtx_off,
                                         const int64_t* edge_off, const ltsnet_params* p,
                                         const ltsnet_batch_config* cfg);
ltsnet_status ltsnet_run_batched(int32_t n_graphs, const int64_t* vtx_off, const int64_t* edge_off,
                                 const int64_t* row_ptr, const int32_t* col, const ltsnet_params* p,
                                 float* Y, void* ws, size_t ws_bytes, const ltsnet_batch_config* cfg,
                                 ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * Pivot MDS initial layout (Alg. 1-3, first step: every variant in the paper
 * starts from a Pivot MDS layout, the method of Brandes and Pich, GD 2006;
 * Sec. 2 names tsNET with this start tsNET*).  The paper fixes none of its
 * parameters; this library takes:
 *  - max-min pivots: pivots[0] = first_pivot; pivot t+1 maximises the BFS
 *    distance to its nearest chosen pivot, the smallest vertex id on ties, a
 *    vertex no chosen pivot reaches counting as infinitely far;
 *  - D = BFS hop distances from the pivots; pairs in different components
 *    take (largest finite distance + 1);
 *  - C = -1/2 J_n (D o D) J_k (double centring, J_m = I - 11^T/m);
 *    x_d = C v_d / sqrt(sigma_d) for the two leading unit eigenvectors v_d of
 *    C^T C (eigenvalues sigma_1^2 >= sigma_2^2), each signed so that its
 *    first entry whose magnitude is within a relative 1e-9 of the largest is
 *    positive; an axis whose eigenvalue is at most 1e-10 of the first is zero;
 *  - one factor on both axes so that the RMS distance from the centroid is
 *    sqrt(2) * init_std (init_std = 1e-4 gives the spread of the random
 *    N(0, 1e-4^2) start); init_std = 0 keeps the MDS scale.
 *   row_ptr, col  graph (device), as everywhere
 *   n_pivots      k, 2 <= k <= min(n, 512); 0 <= first_pivot < n; n >= 2
 *   Y             f32[n][2] (device, out)
 *   pivots        int32[k] (device, out) in the order chosen
 *   dist          uint16[k][n] (device, out, may be NULL): row t holds the
 *                 distances from pivots[t], 0xFFFF where unreached
 *   eigvals       f64[2] (HOST, out, may be NULL): sigma_1^2, sigma_2^2
 * The distance sums behind C^T C are exact integers, so the result does not
 * depend on the order of the GPU's additions.  A BFS distance above 65534
 * returns LTSNET_ERR_INVALID_ARG; a column id outside [0, n) returns
 * LTSNET_ERR_BAD_GRAPH.  Returns LTSNET_WARN_NOT_CONVERGED if the FP64
 * eigen-solve (subspace iteration) stopped at its iteration cap.
 * Synchronous.
 * ------------------------------------------------------------------------- */
size_t ltsnet_pivot_mds_workspace_size(int32_t n, int32_t n_pivots);
ltsnet_status ltsnet_pivot_mds(const int64_t* row_ptr, const int32_t* col, int32_t n, int32_t n_pivots,
                               int32_t first_pivot, double init_std, float* Y, int32_t* pivots,
                               uint16_t* dist, double* eigvals, void* ws, size_t ws_bytes,
                               ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * Quadtree (Barnes-Hut) gradient of BH-tsNET (Alg. 1) and FIt-tsNET (Alg. 2),
 * the paper's other two algorithms, for comparison with L-tsNET.  Same
 * gradient formula as ltsnet_gradient; the attraction A is the exact sparse
 * sum in both variants.
 *   LTSNET_VARIANT_BH:  Z, R and E from the quadtree (BH-SNE's repulsion for
 *                       C1, Eq. 7 for C2).
 *   LTSNET_VARIANT_FIT: A, R, Z and S from ltsnet_gradient's grid
 *                       interpolation (C1), E from the quadtree (C2).
 * The quadtree (the paper leaves its details open): the square at the
 * drawing's minima with side e = the larger extent; depth 16; a point's cell
 * column min(65535, floor((x - lo) * (65536 / e))) in FP32, Morton order;
 * a node of one point is not split; centres of mass exact from fixed point
 * (q = rint((x - lo) 2^36 / e), int64 sums, c = lo + (sum q / |N|) e 2^-36
 * in FP64, rounded to FP32; a one-point node uses the point); a node is a
 * summary for point i if it does not hold i and w^2 < theta^2 d^2 (w = e 2^-l
 * its cell width, d from X_i to its centre, FP32); an opened depth-16 node
 * contributes its points one by one.  theta = 0 gives the exact sums.
 *   grad  f32[n][2] (device); parts f32[n][6] or NULL: (A, R, E) as used;
 *   terms f64[2] (HOST) or NULL: Z, S.
 * Synchronous.  theta >= 0; params as for ltsnet_gradient (only eps is used
 * by the BH variant).
 * ------------------------------------------------------------------------- */
#define LTSNET_VARIANT_BH 1
#define LTSNET_VARIANT_FIT 2
/* The descent loop of Alg. 1 / Alg. 2 with these gradients: the same
 * arguments, schedule, step rule and learning rate as ltsnet_optimize
 * (Y, update, gains f32[n][2] device, in/out), the gradient of each
 * iteration from ltsnet_gradient_quadtree.  Synchronous. */
size_t ltsnet_optimize_quadtree_workspace_size(int32_t n, const ltsnet_params* p, int32_t variant);
ltsnet_status ltsnet_optimize_quadtree(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                                       int32_t n, const ltsnet_params* p, float theta, int32_t variant,
                                       float* Y, float* update, float* gains, int32_t start_iter,
                                       int32_t n_iter, void* ws, size_t ws_bytes, ltsnet_stream stream);
size_t ltsnet_gradient_quadtree_workspace_size(int32_t n, const ltsnet_params* p, int32_t variant);
ltsnet_status ltsnet_gradient_quadtree(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                                       int32_t n, const float* Y, const ltsnet_stage* stage,
                                       const ltsnet_params* p, float theta, int32_t variant, float* grad,
                                       float* parts, double* terms, void* ws, size_t ws_bytes,
                                       ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * Layout quality metrics of Sec. 4 (the paper's NP and ST).  Synchronous.
 * One workspace, ltsnet_quality_workspace_size(n, nnz_graph) bytes (nnz_graph
 * = row_ptr[n], the adjacency entries), serves both calls; the stress call
 * needs only its first part.
 *
 * ltsnet_neighbourhood_preservation -- NP with r = 2: for every vertex v,
 * b = |N_G(v,2)| (vertices within two hops, v excluded), N_D(v) the b
 * vertices nearest to v in the drawing Y (f32[n][2], device), and
 * c = |N_G(v,2) cap N_D(v)|; *np_out (host) = mean of c / (2b - c) over the
 * vertices with b > 0 (the paper prints a sum but states NP lies in [0, 1]),
 * every vertex counted, hubs included.
 * "Nearest" orders (FP32 squared distance, vertex id), the squared distance
 * formed as dx*dx + dy*dy with every operation rounded on its own; ties go to
 * the smaller id.  Balls with more than 2048 two-hop candidates (deg(v) plus
 * the sum of deg(w) over its adjacency entries w) are held in hash tables in
 * the workspace, processed in batches that fit it; LTSNET_ERR_WORKSPACE if one
 * vertex's table does not.
 *   ball, common  int32[n] (device, out, may be NULL): b and c per vertex.
 *
 * ltsnet_stress -- ST: over the ordered pairs (s, j), j != s, for s in
 * sources (int32[n_sources], device), of ((d_sj - alpha ||X_s - X_j||)/d_sj)^2,
 * d the hop distance, at the scale alpha that minimises it (the drawing's
 * scale is free); all vertices as sources give the paper's ST.  Pairs in
 * different components are skipped.  out (host) f64[4]: ST, alpha, pairs
 * counted, pairs skipped.  A BFS distance above 65534 returns
 * LTSNET_ERR_INVALID_ARG; a source out of range too.
 * ------------------------------------------------------------------------- */
size_t ltsnet_quality_workspace_size(int32_t n, int64_t nnz_graph);
ltsnet_status ltsnet_neighbourhood_preservation(const int64_t* row_ptr, const int32_t* col, int32_t n,
                                                const float* Y, int32_t* ball, int32_t* common,
                                                double* np_out, void* ws, size_t ws_bytes,
                                                ltsnet_stream stream);
ltsnet_status ltsnet_stress(const int64_t* row_ptr, const int32_t* col, int32_t n, const float* Y,
                            const int32_t* sources, int32_t n_sources, double* out, void* ws,
                            size_t ws_bytes, ltsnet_stream stream);

/* ---------------------------------------------------------------------------
 * Instrumentation (host side, not part of the method).
 * ltsnet_launch_count: kernels this library has launched in this process.
 * ltsnet_profile_*: times every launch of one kernel with CUDA events on the
 * stream it runs on; `kernel` is one of the LTSNET_KERNEL_* ids.
 * ------------------------------------------------------------------------- */
#define LTSNET_KERNEL_FUSED_UPDATE 1 /* gather + attraction + compression + update */
#define LTSNET_KERNEL_SPREAD 2
#define LTSNET_KERNEL_CONV 3
int64_t ltsnet_launch_count(void);
ltsnet_status ltsnet_profile_begin(int32_t kernel, int32_t max_launches);
ltsnet_status ltsnet_profile_end(int32_t kernel, double* total_ms, int32_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* LTSNET_H */
