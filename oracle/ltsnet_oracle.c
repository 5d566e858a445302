/*
 * FP64 CPU oracle for the L-tsNET gradient hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is built into liboracle.so and is
 * loaded by the tests, by the smoke check and by the benchmark's CPU-baseline
 * leg.  The GPU library never includes, links or calls it, and it includes
 * nothing from the GPU library.
 *
 * Each function restates one step of the method directly from the paper
 * (Meidiana, Hong, Ma, "BH-tsNET, FIt-tsNET, L-tsNET: Fast tsNET Algorithms
 * for Large Graph Drawing"), in double precision, with plain loops and no
 * blocking, fusion or reordering.  Where the paper is silent the reading used
 * is stated beside the code.  Build with -ffp-contract=off so that the FP32
 * grid-rule decisions below round exactly as written.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* C0 step 1: partial BFS (Sec. 3.1, "partial BFS"; Alg. 3 C0 loop).         */
/* From source s run a FIFO breadth-first search over the adjacency lists in  */
/* their stored order.  A vertex counts as visited when it is first reached   */
/* (enqueued).  The search stops the moment k vertices other than s have been */
/* visited.  Reading of "ties are broken randomly": ties are broken by this   */
/* deterministic discovery order.                                             */
/* Outputs for row r = s - s0: nbr[r*k + j] (vertex), hop[r*k + j] (hop       */
/* distance), cnt[r] (number written, = min(k, |component(s)| - 1)); unused   */
/* slots get nbr = -1, hop = 0.                                               */
/* ------------------------------------------------------------------------ */
int or_partial_bfs(int32_t n, const int64_t* row_ptr, const int32_t* col, int32_t k,
                   int32_t s0, int32_t s1, int32_t* nbr, int32_t* hop, int32_t* cnt)
{
    if (n < 0 || k < 1 || s0 < 0 || s1 > n || s0 > s1) return -1;
    int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t* qdist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k + 1));
    if (!mark || !queue || !qdist) { free(mark); free(queue); free(qdist); return -2; }
    for (int32_t v = 0; v < n; ++v) mark[v] = -1;
    for (int32_t s = s0; s < s1; ++s) {
        int64_t r = s - s0;
        int32_t head = 0, tail = 0, found = 0;
        queue[tail] = s; qdist[tail] = 0; ++tail;
        mark[s] = s;
        while (head < tail && found < k) {
            int32_t u = queue[head], du = qdist[head];
            ++head;
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1] && found < k; ++e) {
                int32_t v = col[e];
                if (mark[v] == s) continue;          /* already visited (also s itself) */
                mark[v] = s;
                queue[tail] = v; qdist[tail] = du + 1; ++tail;
                nbr[r * k + found] = v;
                hop[r * k + found] = du + 1;
                ++found;
            }
        }
        cnt[r] = found;
        for (int32_t j = found; j < k; ++j) { nbr[r * k + j] = -1; hop[r * k + j] = 0; }
    }
    free(mark); free(queue); free(qdist);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* C0 step 2: perplexity calibration (Eq. 3 and the perplexity definition    */
/* beneath it).  For row i with neighbours j (hop distance d_ij):            */
/*   p_{j|i}(beta) = exp(-beta d_ij^2) / sum_l exp(-beta d_il^2),            */
/*   beta = 1/(2 sigma_i^2), and beta is chosen so that the entropy          */
/*   H_i = -sum_j p_{j|i} ln p_{j|i} equals ln(u)  (i.e. 2^{H in bits} = u).  */
/* The exponent is shifted by the row's smallest d^2 (this cancels in the    */
/* ratio).  Search (the paper's C0 follows the scikit-learn t-SNE code; the  */
/* paper gives no constants): start at beta = 1; if H is above the target    */
/* raise beta (double while no upper bound is known, else bisect), otherwise */
/* lower it (halve while no lower bound is known, else bisect); stop when    */
/* |H - ln u| < tol or after max_steps evaluations.  The output p is         */
/* evaluated at the final beta.  converged[i] = 1 iff the tolerance was met. */
/* Rows with no neighbours get beta = 1, converged = 0.                      */
/* ------------------------------------------------------------------------ */
static void or_row_probs(int32_t c, const int32_t* hop, double beta, double* p)
{
    double dmin = INFINITY;
    for (int32_t j = 0; j < c; ++j) {
        double d2 = (double)hop[j] * (double)hop[j];
        if (d2 < dmin) dmin = d2;
    }
    double sum = 0.0;
    for (int32_t j = 0; j < c; ++j) {
        double d2 = (double)hop[j] * (double)hop[j];
        p[j] = exp(-beta * (d2 - dmin));
        sum += p[j];
    }
    for (int32_t j = 0; j < c; ++j) p[j] /= sum;
}

static double or_entropy(int32_t c, const double* p)
{
    double h = 0.0;
    for (int32_t j = 0; j < c; ++j)
        if (p[j] > 0.0) h -= p[j] * log(p[j]);
    return h;
}

int or_calibrate(int32_t n, int32_t k, const int32_t* hop, const int32_t* cnt,
                 double perplexity, double tol, int32_t max_steps,
                 double* beta_out, double* pcond, uint8_t* converged)
{
    if (n < 0 || k < 1 || !(perplexity > 0.0)) return -1;
    double target = log(perplexity);
    double* p = (double*)malloc(sizeof(double) * (size_t)k);
    if (!p) return -2;
    for (int32_t i = 0; i < n; ++i) {
        int32_t c = cnt[i];
        const int32_t* h = hop + (int64_t)i * k;
        double beta = 1.0, lo = -INFINITY, hi = INFINITY;
        int ok = 0;
        if (c > 0) {
            for (int32_t step = 0; step < max_steps; ++step) {
                or_row_probs(c, h, beta, p);
                double diff = or_entropy(c, p) - target;
                if (fabs(diff) < tol) { ok = 1; break; }
                if (diff > 0.0) {
                    lo = beta;
                    beta = (hi == INFINITY) ? beta * 2.0 : (beta + hi) / 2.0;
                } else {
                    hi = beta;
                    beta = (lo == -INFINITY) ? beta / 2.0 : (beta + lo) / 2.0;
                }
            }
            or_row_probs(c, h, beta, p);
        }
        beta_out[i] = beta;
        converged[i] = (uint8_t)ok;
        for (int32_t j = 0; j < k; ++j) pcond[(int64_t)i * k + j] = (j < c) ? p[j] : 0.0;
    }
    free(p);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* C0 step 3: symmetrisation (Eq. 2).  p_ij = (p_{j|i} + p_{i|j}) / (2n)     */
/* over the union of both supports (a missing conditional counts as zero).   */
/* Output: CSR with each row's columns ascending.  P_val64 holds the FP64    */
/* value; callers round it to FP32 themselves.  Returns nnz, or -1 if `cap`  */
/* is too small, -2 on allocation failure.                                   */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t col; double val; } or_entry;

static int or_entry_cmp(const void* a, const void* b)
{
    int32_t x = ((const or_entry*)a)->col, y = ((const or_entry*)b)->col;
    return (x > y) - (x < y);
}

int64_t or_symmetrize(int32_t n, int32_t k, const int32_t* nbr, const int32_t* cnt,
                      const double* pcond, int64_t* P_row, int32_t* P_col,
                      double* P_val64, int64_t cap)
{
    /* rows of the transposed conditional matrix: tr[i] lists (j, p_{i|j}) */
    int64_t* tcount = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!tcount) return -2;
    for (int32_t j = 0; j < n; ++j)
        for (int32_t s = 0; s < cnt[j]; ++s) tcount[nbr[(int64_t)j * k + s] + 1]++;
    for (int32_t i = 0; i < n; ++i) tcount[i + 1] += tcount[i];
    int64_t total_t = tcount[n];
    or_entry* tr = (or_entry*)malloc(sizeof(or_entry) * (size_t)(total_t > 0 ? total_t : 1));
    int64_t* fillp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    or_entry* rowbuf = (or_entry*)malloc(sizeof(or_entry) * (size_t)(total_t + k + 1));
    if (!tr || !fillp || !rowbuf) { free(tcount); free(tr); free(fillp); free(rowbuf); return -2; }
    for (int32_t i = 0; i < n; ++i) fillp[i] = tcount[i];
    for (int32_t j = 0; j < n; ++j)
        for (int32_t s = 0; s < cnt[j]; ++s) {
            int32_t i = nbr[(int64_t)j * k + s];
            tr[fillp[i]].col = j;
            tr[fillp[i]].val = pcond[(int64_t)j * k + s];
            fillp[i]++;
        }
    const double inv2n = 1.0 / (2.0 * (double)n);
    int64_t nnz = 0;
    P_row[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t len = 0;
        for (int32_t s = 0; s < cnt[i]; ++s) {
            rowbuf[len].col = nbr[(int64_t)i * k + s];
            rowbuf[len].val = pcond[(int64_t)i * k + s];
            ++len;
        }
        for (int64_t t = tcount[i]; t < tcount[i + 1]; ++t) rowbuf[len++] = tr[t];
        qsort(rowbuf, (size_t)len, sizeof(or_entry), or_entry_cmp);
        for (int64_t t = 0; t < len;) {
            int32_t c = rowbuf[t].col;
            double v = 0.0;
            while (t < len && rowbuf[t].col == c) { v += rowbuf[t].val; ++t; }
            if (nnz >= cap) { free(tcount); free(tr); free(fillp); free(rowbuf); return -1; }
            P_col[nnz] = c;
            P_val64[nnz] = v * inv2n;
            ++nnz;
        }
        P_row[i + 1] = nnz;
    }
    free(tcount); free(tr); free(fillp); free(rowbuf);
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* EXACT per-iteration terms (Eq. 1, Eq. 6, the q_ij definition in Sec. 2.1  */
/* and the L-tsNET entropy kernel of Sec. 3.3), O(n^2), FP64:                */
/*   K1 = 1/(1+d^2), K2 = K1^2, Ke = 1/(eps + d^2), d = |X_i - X_j|           */
/*   Z      = sum_{i != j} K1                                                 */
/*   A_i    = sum_{j in row i of P} p_ij K1 (X_i - X_j)      (attraction)     */
/*   R_i    = sum_{j != i} K2 (X_i - X_j)                     (repulsion)     */
/*   E_i    = sum_{j != i} Ke (X_i - X_j)                     (entropy)       */
/* Outputs are the unscaled sums; callers assemble the gradient.             */
/* ------------------------------------------------------------------------ */
int or_exact_sums(int32_t n, const double* Y, const int64_t* P_row, const int32_t* P_col,
                  const double* P_val, double eps, double* A, double* R, double* E, double* Z_out)
{
    double Z = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double xi = Y[2 * i], yi = Y[2 * i + 1];
        double rx = 0, ry = 0, ex = 0, ey = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = xi - Y[2 * j], dy = yi - Y[2 * j + 1];
            double d2 = dx * dx + dy * dy;
            double k1 = 1.0 / (1.0 + d2);
            double ke = 1.0 / (eps + d2);
            Z += k1;
            rx += k1 * k1 * dx; ry += k1 * k1 * dy;
            ex += ke * dx; ey += ke * dy;
        }
        double ax = 0, ay = 0;
        for (int64_t e = P_row[i]; e < P_row[i + 1]; ++e) {
            int32_t j = P_col[e];
            double dx = xi - Y[2 * j], dy = yi - Y[2 * j + 1];
            double k1 = 1.0 / (1.0 + dx * dx + dy * dy);
            ax += P_val[e] * k1 * dx; ay += P_val[e] * k1 * dy;
        }
        A[2 * i] = ax; A[2 * i + 1] = ay;
        R[2 * i] = rx; R[2 * i + 1] = ry;
        E[2 * i] = ex; E[2 * i + 1] = ey;
    }
    *Z_out = Z;
    return 0;
}

/* EXACT cost pieces (Eq. 1 with the KL term of Eq. 4 and q_ij of Sec. 2.1). */
/*   out[0] = sum_e p_e ln p_e                                                */
/*   out[1] = sum_e p_e ln(1 + d_e^2)                                         */
/*   out[2] = Z = sum_{i != j} 1/(1 + d^2)                                    */
/*   out[3] = sum_i |X_i|^2                                                   */
/*   out[4] = sum_{i != j} ln(eps + d^2)   (the entropy reading)              */
/*   out[5] = sum_{i != j} ln(d)           (the paper's literal form, eps=0)  */
/*   out[6] = S = sum_e p_e                                                   */
int or_exact_cost_parts(int32_t n, const double* Y, const int64_t* P_row, const int32_t* P_col,
                        const double* P_val, double eps, double* out)
{
    double plogp = 0, plogk = 0, Z = 0, sq = 0, lent = 0, llit = 0, S = 0;
    for (int32_t i = 0; i < n; ++i) {
        double xi = Y[2 * i], yi = Y[2 * i + 1];
        sq += xi * xi + yi * yi;
        for (int32_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = xi - Y[2 * j], dy = yi - Y[2 * j + 1];
            double d2 = dx * dx + dy * dy;
            Z += 1.0 / (1.0 + d2);
            lent += log(eps + d2);
            llit += 0.5 * log(d2);
        }
        for (int64_t e = P_row[i]; e < P_row[i + 1]; ++e) {
            int32_t j = P_col[e];
            double dx = xi - Y[2 * j], dy = yi - Y[2 * j + 1];
            double p = P_val[e];
            S += p;
            if (p > 0) plogp += p * log(p);
            plogk += p * log(1.0 + dx * dx + dy * dy);
        }
    }
    out[0] = plogp; out[1] = plogk; out[2] = Z; out[3] = sq; out[4] = lent; out[5] = llit; out[6] = S;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* INTERP: the L-tsNET interpolation (Sec. 2.3 "four sums", Sec. 3.3 h1..h3, */
/* Alg. 3 loop).  The grid constants are not in the paper; the reading:      */
/* one square domain [lo, lo+ext] with lo/hi the min/max over all x and y    */
/* coordinates, I boxes per dimension, nodes_per_box (P) Lagrange nodes per  */
/* box at the box's cell centres.  The integer decisions (I, box index) are  */
/* taken in FP32 exactly as the GPU takes them, so both sides choose the     */
/* same boxes.                                                               */
/* ------------------------------------------------------------------------ */
static int or_is_smooth(int32_t v)
{
    if (v < 1) return 0;
    while (v % 2 == 0) v /= 2;
    while (v % 3 == 0) v /= 3;
    while (v % 5 == 0) v /= 5;
    return v == 1;
}

/* grid[0]=lo, grid[1]=hi, grid[2]=ext, grid[3]=h, grid[4]=s (node spacing),  */
/* grid[5]=centre; igrid[0]=I, igrid[1]=M = I*P                              */
int or_grid_rule(int32_t n, const float* Y, float box_width_max, int32_t min_boxes,
                 int32_t max_boxes, int32_t nodes_per_box, float* grid, int32_t* igrid)
{
    if (n < 1 || !(box_width_max > 0.0f) || min_boxes < 1 || max_boxes < min_boxes || nodes_per_box < 1)
        return -1;
    float lo = Y[0], hi = Y[0];
    for (int64_t t = 0; t < 2 * (int64_t)n; ++t) {
        float v = Y[t];
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    float ext = hi - lo;
    if (!(ext >= 1e-6f)) ext = 1e-6f;
    float q = ext / box_width_max;
    int32_t I;
    if (!(q < (float)max_boxes)) I = max_boxes;
    else I = (int32_t)ceilf(q);
    if (I < min_boxes) I = min_boxes;
    while (!or_is_smooth(I)) ++I;
    if (I > max_boxes) {
        I = max_boxes;
        while (I > 1 && !or_is_smooth(I)) --I;
    }
    float h = ext / (float)I;
    float s = h / (float)nodes_per_box;
    float c = 0.5f * (lo + hi);
    grid[0] = lo; grid[1] = hi; grid[2] = ext; grid[3] = h; grid[4] = s; grid[5] = c;
    igrid[0] = I; igrid[1] = I * nodes_per_box;
    return 0;
}

static int32_t or_box(float x, float lo, float h, int32_t I)
{
    float t = (x - lo) / h;
    int32_t b = (int32_t)floorf(t);
    if (b < 0) b = 0;
    if (b > I - 1) b = I - 1;
    return b;
}

/* Lagrange weights of x for the P nodes of its box: nodes at local          */
/* coordinates u_a = a + 1/2 (in units of the node spacing s).               */
static void or_lagrange(double x, double lo, double s, int32_t b, int32_t P, double* w)
{
    double u = (x - lo) / s - (double)P * (double)b;
    for (int32_t a = 0; a < P; ++a) {
        double num = 1.0, den = 1.0;
        for (int32_t c = 0; c < P; ++c) {
            if (c == a) continue;
            num *= u - ((double)c + 0.5);
            den *= ((double)a + 0.5) - ((double)c + 0.5);
        }
        w[a] = num / den;
    }
}

/* Spread: W_c[ty*M + tx] = sum_i L_tx(x_i) L_ty(y_i) q_c(i), charges          */
/* q = (1, x~, y~, x~^2 + y~^2) in coordinates centred at `centre`.           */
/* W has 4*M*M doubles, charge-major.  box_out (optional) gets (bx, by).      */
int or_spread(int32_t n, const float* Y, const float* grid, const int32_t* igrid,
              int32_t P, double* W, int32_t* box_out)
{
    float lo = grid[0], h = grid[3];
    double s = (double)grid[4], c = (double)grid[5];
    int32_t I = igrid[0], M = igrid[1];
    if (P > 16) return -1;
    memset(W, 0, sizeof(double) * 4 * (size_t)M * (size_t)M);
    double wx[16], wy[16];
    for (int32_t i = 0; i < n; ++i) {
        float x = Y[2 * i], y = Y[2 * i + 1];
        int32_t bx = or_box(x, lo, h, I), by = or_box(y, lo, h, I);
        if (box_out) { box_out[2 * i] = bx; box_out[2 * i + 1] = by; }
        or_lagrange((double)x, (double)lo, s, bx, P, wx);
        or_lagrange((double)y, (double)lo, s, by, P, wy);
        double xt = (double)x - c, yt = (double)y - c;
        double q[4] = {1.0, xt, yt, xt * xt + yt * yt};
        for (int32_t b = 0; b < P; ++b)
            for (int32_t a = 0; a < P; ++a) {
                int64_t node = (int64_t)(P * by + b) * M + (P * bx + a);
                double w = wx[a] * wy[b];
                for (int32_t ch = 0; ch < 4; ++ch) W[(int64_t)ch * M * M + node] += w * q[ch];
            }
    }
    return 0;
}

/* Direct convolution on the node grid (O(M^4); small M only):              */
/*   phi_c[t] = sum_t' K2(xi_t - xi_t') W_c[t']   c = 0..3                  */
/*   hfl_c[t] = sum_t' Ke(xi_t - xi_t') W_c[t']   c = 0..2                  */
/* out has 7*M*M doubles in the order phi0..phi3, h1, h2, h3.               */
int or_conv_direct(int32_t M, double s, double eps, const double* W, double* out)
{
    int64_t MM = (int64_t)M * M;
    memset(out, 0, sizeof(double) * 7 * (size_t)MM);
    for (int32_t ty = 0; ty < M; ++ty)
        for (int32_t tx = 0; tx < M; ++tx) {
            double acc[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int32_t uy = 0; uy < M; ++uy)
                for (int32_t ux = 0; ux < M; ++ux) {
                    double dx = s * (double)(tx - ux), dy = s * (double)(ty - uy);
                    double d2 = dx * dx + dy * dy;
                    double k1 = 1.0 / (1.0 + d2);
                    double k2 = k1 * k1, ke = 1.0 / (eps + d2);
                    int64_t src = (int64_t)uy * M + ux;
                    for (int32_t ch = 0; ch < 4; ++ch) acc[ch] += k2 * W[ch * MM + src];
                    for (int32_t ch = 0; ch < 3; ++ch) acc[4 + ch] += ke * W[ch * MM + src];
                }
            for (int32_t f = 0; f < 7; ++f) out[f * MM + (int64_t)ty * M + tx] = acc[f];
        }
    return 0;
}

/* Gather: Phi_f(i) = sum_{a,b} L_a(x_i) L_b(y_i) fld_f[node(a,b)], f = 0..6. */
int or_gather(int32_t n, const float* Y, const float* grid, const int32_t* igrid, int32_t P,
              const double* fld, double* Phi)
{
    float lo = grid[0], h = grid[3];
    double s = (double)grid[4];
    int32_t I = igrid[0], M = igrid[1];
    int64_t MM = (int64_t)M * M;
    if (P > 16) return -1;
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double wx[16], wy[16];
        float x = Y[2 * i], y = Y[2 * i + 1];
        int32_t bx = or_box(x, lo, h, I), by = or_box(y, lo, h, I);
        or_lagrange((double)x, (double)lo, s, bx, P, wx);
        or_lagrange((double)y, (double)lo, s, by, P, wy);
        double acc[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int32_t b = 0; b < P; ++b)
            for (int32_t a = 0; a < P; ++a) {
                int64_t node = (int64_t)(P * by + b) * M + (P * bx + a);
                double w = wx[a] * wy[b];
                for (int32_t f = 0; f < 7; ++f) acc[f] += w * fld[f * MM + node];
            }
        for (int32_t f = 0; f < 7; ++f) Phi[(int64_t)i * 7 + f] = acc[f];
    }
    return 0;
}

/* Attractive sum A_i = sum_{j in row i} p_ij (X_i - X_j)/(1 + |X_i - X_j|^2) */
/* (first term of Eq. 6), on the FP32 layout read as doubles.                */
int or_attractive(int32_t n, const float* Y, const int64_t* P_row, const int32_t* P_col,
                  const double* P_val, double* A)
{
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double xi = Y[2 * i], yi = Y[2 * i + 1], ax = 0, ay = 0;
        for (int64_t e = P_row[i]; e < P_row[i + 1]; ++e) {
            int32_t j = P_col[e];
            double dx = xi - (double)Y[2 * j], dy = yi - (double)Y[2 * j + 1];
            double k1 = 1.0 / (1.0 + dx * dx + dy * dy);
            ax += P_val[e] * k1 * dx; ay += P_val[e] * k1 * dy;
        }
        A[2 * i] = ax; A[2 * i + 1] = ay;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* EXACT sums of or_exact_sums for selected target rows only (A_i, R_i, E_i   */
/* over every source j != i, Eq. 6 and the Sec. 3.3 kernel), for sampled     */
/* checks of layouts too large for the O(n^2) pass over all rows.  Output    */
/* row r belongs to vertex rows[r].  Each row is summed by one thread in     */
/* source order (OpenMP over the listed rows when built with -fopenmp), so    */
/* the result does not depend on the thread count.                            */
/* ------------------------------------------------------------------------ */
int or_exact_rows(int32_t n, const double* Y, const int64_t* P_row, const int32_t* P_col,
                  const double* P_val, double eps, int32_t nrows, const int32_t* rows,
                  double* A, double* R, double* E)
{
    for (int32_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= n) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t r = 0; r < nrows; ++r) {
        int32_t i = rows[r];
        double xi = Y[2 * i], yi = Y[2 * i + 1];
        double rx = 0, ry = 0, ex = 0, ey = 0, ax = 0, ay = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = xi - Y[2 * j], dy = yi - Y[2 * j + 1];
            double d2 = dx * dx + dy * dy;
            double k1 = 1.0 / (1.0 + d2);
            double ke = 1.0 / (eps + d2);
            rx += k1 * k1 * dx; ry += k1 * k1 * dy;
            ex += ke * dx; ey += ke * dy;
        }
        for (int64_t e = P_row[i]; e < P_row[i + 1]; ++e) {
            int32_t j = P_col[e];
            double dx = xi - Y[2 * j], dy = yi - Y[2 * j + 1];
            double k1 = 1.0 / (1.0 + dx * dx + dy * dy);
            ax += P_val[e] * k1 * dx; ay += P_val[e] * k1 * dy;
        }
        A[2 * r] = ax; A[2 * r + 1] = ay;
        R[2 * r] = rx; R[2 * r + 1] = ry;
        E[2 * r] = ex; E[2 * r + 1] = ey;
    }
    return 0;
}

/* Z = sum_{i != j} 1/(1 + |X_i - X_j|^2) (the normalisation of q_ij, Sec.   */
/* 2.1 and Eq. 6): row sums in source order (OpenMP over rows), then the row  */
/* sums added in row order.                                                   */
int or_exact_z(int32_t n, const double* Y, double* Z_out)
{
    double* rs = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!rs) return -2;
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t i = 0; i < n; ++i) {
        double xi = Y[2 * i], yi = Y[2 * i + 1], z = 0.0;
        for (int32_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = xi - Y[2 * j], dy = yi - Y[2 * j + 1];
            z += 1.0 / (1.0 + dx * dx + dy * dy);
        }
        rs[i] = z;
    }
    double Z = 0.0;
    for (int32_t i = 0; i < n; ++i) Z += rs[i];
    free(rs);
    *Z_out = Z;
    return 0;
}

/* Change of the EXACT cost's pieces (or_exact_cost_parts) when coordinate d  */
/* (0 = x, 1 = y) of vertex i moves by +h and by -h, from only the terms that */
/* involve i, so that central differences of the cost need O(n + nnz) work:   */
/*   out[0] = sum over entries e touching i (row i and column i) of           */
/*            p_e [ln(1 + d_e+^2) - ln(1 + d_e-^2)]                           */
/*   out[1] = Z(+h) - Z,  out[2] = Z(-h) - Z  (ordered pairs, i on either side) */
/*   out[3] = sum_{i != j} ln(eps + d^2) at +h minus at -h (both orders)       */
/*   out[4] = |X|^2 at +h minus at -h                                          */
/* The cost at +h minus the cost at -h is then                                 */
/*   l_KL [out0 + S (ln(Z + out1) - ln(Z + out2))] + l_c/(2n) out4             */
/*   - l_r/(4n^2) out3.                                                        */
int or_exact_cost_step(int32_t n, const double* Y, const int64_t* P_row, const int32_t* P_col,
                       const double* P_val, double eps, int32_t i, int32_t d, double h, double* out)
{
    if (i < 0 || i >= n || d < 0 || d > 1) return -1;
    double xp[2] = {Y[2 * i], Y[2 * i + 1]}, xm[2] = {Y[2 * i], Y[2 * i + 1]}, x0[2] = {Y[2 * i], Y[2 * i + 1]};
    xp[d] += h;
    xm[d] -= h;
    double kl = 0.0, zp = 0.0, zm = 0.0, le = 0.0;
    for (int32_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double yj0 = Y[2 * j], yj1 = Y[2 * j + 1];
        double ap = xp[0] - yj0, bp = xp[1] - yj1, am = xm[0] - yj0, bm = xm[1] - yj1;
        double a0 = x0[0] - yj0, b0 = x0[1] - yj1;
        double d2p = ap * ap + bp * bp, d2m = am * am + bm * bm, d20 = a0 * a0 + b0 * b0;
        double k0 = 1.0 / (1.0 + d20);
        zp += 2.0 * (1.0 / (1.0 + d2p) - k0);
        zm += 2.0 * (1.0 / (1.0 + d2m) - k0);
        le += 2.0 * (log(eps + d2p) - log(eps + d2m));
    }
    for (int32_t r = 0; r < n; ++r)
        for (int64_t e = P_row[r]; e < P_row[r + 1]; ++e) {
            int32_t c = P_col[e];
            if (r != i && c != i) continue;
            if (r == i && c == i) continue; /* a self entry has d = 0 either way */
            int32_t j = r == i ? c : r;
            double ap = xp[0] - Y[2 * j], bp = xp[1] - Y[2 * j + 1];
            double am = xm[0] - Y[2 * j], bm = xm[1] - Y[2 * j + 1];
            kl += P_val[e] * (log(1.0 + ap * ap + bp * bp) - log(1.0 + am * am + bm * bm));
        }
    out[0] = kl;
    out[1] = zp;
    out[2] = zm;
    out[3] = le;
    out[4] = xp[d] * xp[d] - xm[d] * xm[d];
    return 0;
}

/* Threads for the row-parallel loops (each row is summed by one thread in a  */
/* fixed order, so results do not depend on the count); returns the count in  */
/* use, 1 without OpenMP.                                                     */
int or_set_threads(int32_t t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}
