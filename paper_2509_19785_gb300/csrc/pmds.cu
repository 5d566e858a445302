// Pivot MDS initial layout: the first step of Alg. 1-3 ("compute the initial
// layout with Pivot MDS"; the paper takes the method from Brandes and Pich,
// GD 2006, and gives none of its parameters).
//
//  1. Max-min pivots.  Pivot 0 is given; pivot t+1 is the vertex whose BFS
//     distance to its nearest chosen pivot is largest, the smallest index on
//     ties, a vertex no pivot reaches counting as infinitely far.
//  2. D: hop distances from every pivot, one uint16 row of n per pivot
//     (0xFFFF = unreached), by the level-synchronous BFS of bfs_levels.cuh.
//  3. A = D o D with unreached pairs at (largest finite distance + 1);
//     C = -1/2 J_n A J_k.  Then C^T C = 1/4 J_k (G - s s^T / n) J_k with
//     G = A^T A and s = A^T 1.  G and s are sums of integers, accumulated
//     exactly (128-bit for G), so they do not depend on the order of the
//     additions.
//  4. The two leading eigenpairs (sigma_d^2, v_d) of C^T C: subspace
//     iteration with a Rayleigh-Ritz step, in FP64, in one block.
//  5. x_d = C v_d / sqrt(sigma_d) = A w_d - o_d with
//     w_d = -1/2 J_k v_d / sqrt(sigma_d) and o_d = s^T w_d / n (FP64), then
//     one factor on both axes so that the RMS distance from the centroid is
//     sqrt(2) init_std.
//
// The scale 1/sqrt(sigma_d) makes the method classical MDS when every
// vertex is a pivot.  Each v_d is signed so that its first entry whose
// magnitude is within a relative 1e-9 of the largest is positive (the slack
// keeps the choice stable under rounding where entries tie in magnitude); an
// axis whose eigenvalue is at most 1e-10 of the first is zero.
#include <math.h>

#include <algorithm>

#include "bfs_levels.cuh"

namespace lt {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxPivots = 512;
constexpr int kTile = 64;         // pivots per side of a Gram tile
constexpr int kRows = 64;         // rows staged per step of the Gram kernel
constexpr int kPad = 68;          // words per staged column: 16-byte aligned, spreads the banks
constexpr int kRitz = 4;          // subspace dimension of the eigen-solve
constexpr int kEigMaxIter = 20000;
constexpr double kEigTol = 1e-13;
constexpr double kAxisEps = 1e-10;
constexpr double kSignSlack = 1e-9;
constexpr int kFlatBlocks = kSplitBlocks * 4;  // fixed: sizes workspace partials

struct PmdsEig {
    double lam[2];   // sigma_d^2
    double o[2];
    int32_t iters;
    int32_t converged;
    int32_t pad[2];
};

__device__ __forceinline__ uint32_t sq_dist(uint16_t d, uint32_t fill)
{
    const uint32_t v = d == kUnreached ? fill : (uint32_t)d;
    return v * v;  // fill <= 65535
}

// ---------------------------------------------------------------------------
// Step 1-2: pivots and BFS rows.

__global__ void k_pmds_pivot(int32_t t, int32_t first, int32_t n, const unsigned long long* __restrict__ best,
                             int32_t* __restrict__ pivots, uint16_t* __restrict__ D, int32_t* __restrict__ q0,
                             LevelCtl* ctl, StatusBlock* st)
{
    int32_t p = first;
    if (t > 0) p = (int32_t)(0xFFFFFFFFu - (uint32_t)(best[t] & 0xFFFFFFFFull));
    if (p < 0 || p >= n) {  // cannot happen for 2 <= k <= n; kept as a guard
        record_error(st, LTSNET_ERR_INVALID_ARG, t);
        ctl->cnt[0] = ctl->cnt[1] = 0;
        ctl->err = 3;
        return;
    }
    pivots[t] = p;
    bfs_seed(ctl, D, n, t, p, q0);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

// After pivot t's BFS: nearest[v] = min(nearest[v], d_t(v)); the next pivot
// is the largest key (nearest << 32 | ~v), i.e. the largest nearest distance
// with the smallest index; dmax tracks the largest finite distance.
__global__ void __launch_bounds__(kThreads) k_pmds_nearest(const uint16_t* __restrict__ D, int32_t t, int32_t n,
                                                           uint32_t* __restrict__ nearest,
                                                           unsigned long long* __restrict__ best_next,
                                                           int32_t* __restrict__ dmax)
{
    const uint16_t* d = D + (size_t)t * n;
    unsigned long long key = 0;
    int32_t fmax = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t dv = d[v];
        uint32_t dd = 0xFFFFFFFFu;
        if (dv != kUnreached) {
            dd = dv;
            fmax = max(fmax, (int32_t)dv);
        }
        const uint32_t nv = min(nearest[v], dd);
        nearest[v] = nv;
        key = umax64(key, ((unsigned long long)nv << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)v));
    }
    __shared__ unsigned long long skey[kThreads / 32];
    __shared__ int32_t smax[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        key = umax64(key, __shfl_xor_sync(FULL, key, o));
        fmax = max(fmax, __shfl_xor_sync(FULL, fmax, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        skey[w] = key;
        smax[w] = fmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kThreads / 32; ++i) {
            key = umax64(key, skey[i]);
            fmax = max(fmax, smax[i]);
        }
        if (best_next) atomicMax(best_next, key);
        atomicMax(dmax, fmax);
    }
}

// ---------------------------------------------------------------------------
// Step 3: s = A^T 1 and G = A^T A, exact.

__global__ void __launch_bounds__(kThreads) k_pmds_colsum(const uint16_t* __restrict__ D, int32_t n,
                                                          const int32_t* __restrict__ dmax,
                                                          unsigned long long* __restrict__ colsum)
{
    const uint32_t fill = (uint32_t)*dmax + 1u;
    const uint16_t* d = D + (size_t)blockIdx.y * n;
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += sq_dist(d[i], fill);
    acc = warp_sum(acc);
    __shared__ unsigned long long red[kThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kThreads / 32; ++i) acc += red[i];
        atomicAdd(&colsum[blockIdx.y], acc);
    }
}

__device__ __forceinline__ void mac128(unsigned long long& lo, unsigned long long& hi, uint32_t a, uint32_t b)
{
    const unsigned long long p = (unsigned long long)a * b;
    lo += p;
    hi += lo < p ? 1ull : 0ull;
}

// 128-bit add into G[2 idx] (low word), G[2 idx + 1] (high word).  The high
// word takes one carry for every wrap of the low word, so the final pair is
// the exact sum whatever the order of the blocks.
__device__ __forceinline__ void add128(unsigned long long* G, size_t idx, unsigned long long lo, unsigned long long hi)
{
    const unsigned long long old = atomicAdd(&G[2 * idx], lo);
    const unsigned long long carry = old + lo < old ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&G[2 * idx + 1], hi + carry);
}

// One 64 x 64 tile (pivot blocks tb_j <= tb_l) of G over one range of rows.
// Thread (tj, tl) owns pivots j = 64 tb_j + tj + 16a and l = 64 tb_l + tl + 16c
// (a, c = 0..3).  Squared distances are staged column-wise in shared memory.
__global__ void __launch_bounds__(kThreads) k_pmds_gram(const uint16_t* __restrict__ D, int32_t n, int32_t k,
                                                        int32_t rows_per_block, const int32_t* __restrict__ dmax,
                                                        unsigned long long* __restrict__ G)
{
    __shared__ __align__(16) uint32_t Sj[kTile][kPad];
    __shared__ __align__(16) uint32_t Sl[kTile][kPad];
    const int ntb = (k + kTile - 1) / kTile;
    int q = blockIdx.x, tbj = 0;
    while (q >= ntb - tbj) {
        q -= ntb - tbj;
        ++tbj;
    }
    const int tbl = tbj + q;
    const uint32_t fill = (uint32_t)*dmax + 1u;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
    const int64_t r1 = min((int64_t)n, r0 + rows_per_block);
    const int tj = threadIdx.x >> 4, tl = threadIdx.x & 15;
    unsigned long long lo[4][4], hi[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) lo[a][c] = hi[a][c] = 0;
    for (int64_t rb = r0; rb < r1; rb += kRows) {
        __syncthreads();
        for (int e = threadIdx.x; e < kTile * kRows; e += kThreads) {
            const int c = e / kRows, r = e % kRows;
            const int64_t i = rb + r;
            const int jj = tbj * kTile + c, ll = tbl * kTile + c;
            uint32_t vj = 0, vl = 0;
            if (i < r1) {
                if (jj < k) vj = sq_dist(D[(size_t)jj * n + i], fill);
                if (ll < k) vl = sq_dist(D[(size_t)ll * n + i], fill);
            }
            Sj[c][r] = vj;
            Sl[c][r] = vl;
        }
        __syncthreads();
#pragma unroll 1
        for (int r = 0; r < kRows; r += 4) {
            uint4 av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = *reinterpret_cast<const uint4*>(&Sj[tj + 16 * a][r]);
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = *reinterpret_cast<const uint4*>(&Sl[tl + 16 * c][r]);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    mac128(lo[a][c], hi[a][c], av[a].x, bv[c].x);
                    mac128(lo[a][c], hi[a][c], av[a].y, bv[c].y);
                    mac128(lo[a][c], hi[a][c], av[a].z, bv[c].z);
                    mac128(lo[a][c], hi[a][c], av[a].w, bv[c].w);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = tbj * kTile + tj + 16 * a, l = tbl * kTile + tl + 16 * c;
            if (j < k && l < k && (tbj < tbl || j <= l) && (lo[a][c] | hi[a][c]))
                add128(G, (size_t)j * k + l, lo[a][c], hi[a][c]);
        }
}

// ---------------------------------------------------------------------------
// Step 4: eigen-solve, one block.

// Sum over the block of R values per thread; every thread gets the totals.
// The order of the additions is fixed, so the result is reproducible.
template <int R>
__device__ void block_sums(double (&v)[R], double (*red)[R])
{
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = warp_sum(v[i]);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < R; ++i) red[w][i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i) {
        double s = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) s += red[q][i];
        v[i] = s;
    }
    __syncthreads();
}

// Deterministic start vectors in [-1, 1): a 64-bit integer hash of (j, c, salt).
__device__ double start_value(int j, int c, int salt)
{
    unsigned long long x = ((unsigned long long)(j + 1) << 20) ^ ((unsigned long long)(c + 1) << 8) ^ (unsigned long long)salt;
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return (double)(x >> 11) * 0x1p-52 - 1.0;
}

struct EigSmem {
    double Q[kMaxPivots][kRitz];
    double Z[kMaxPivots][kRitz];
    double red[kThreads / 32][kRitz * kRitz];
    double T[kRitz][kRitz];
    double U[kRitz][kRitz];
    double lam[kRitz];
    double scal[4];
    int32_t flag;
};

// Modified Gram-Schmidt, twice, on the columns of Q (rows k).  A column that
// loses all but 1e-10 of its norm to the projections (it lies in the span of
// the earlier ones, e.g. M of rank below r) is replaced by a fresh start
// vector and orthogonalised again.
__device__ void orthonormalise(EigSmem& S, int k, int r, int salt)
{
    double (*red1)[1] = reinterpret_cast<double (*)[1]>(&S.red[0][0]);
    double (*red3)[3] = reinterpret_cast<double (*)[3]>(&S.red[0][0]);
    for (int c = 0; c < r; ++c) {
        for (int attempt = 0; attempt < 4; ++attempt) {
            double n0[1] = {0.0};
            for (int j = threadIdx.x; j < k; j += kThreads) n0[0] += S.Q[j][c] * S.Q[j][c];
            block_sums<1>(n0, red1);
            for (int pass = 0; pass < 2 && c > 0; ++pass) {
                double dots[3] = {0.0, 0.0, 0.0};
                for (int j = threadIdx.x; j < k; j += kThreads)
                    for (int p = 0; p < c; ++p) dots[p] += S.Q[j][p] * S.Q[j][c];
                block_sums<3>(dots, red3);
                for (int j = threadIdx.x; j < k; j += kThreads) {
                    double x = S.Q[j][c];
                    for (int p = 0; p < c; ++p) x -= dots[p] * S.Q[j][p];
                    S.Q[j][c] = x;
                }
                __syncthreads();
            }
            double nn[1] = {0.0};
            for (int j = threadIdx.x; j < k; j += kThreads) nn[0] += S.Q[j][c] * S.Q[j][c];
            block_sums<1>(nn, red1);
            const double nrm = sqrt(nn[0]);
            if (nrm > 1e-10 * sqrt(n0[0]) && nrm > 0.0) {
                const double inv = 1.0 / nrm;
                for (int j = threadIdx.x; j < k; j += kThreads) S.Q[j][c] *= inv;
                __syncthreads();
                break;
            }
            for (int j = threadIdx.x; j < k; j += kThreads) S.Q[j][c] = start_value(j, c, salt + 17 * (attempt + 1));
            __syncthreads();
        }
    }
}

// Cyclic Jacobi rotations on the symmetric r x r matrix T (thread 0):
// T = U diag(lam) U^T, eigenvalues sorted descending.
__device__ void small_eigen(EigSmem& S, int r)
{
    double A[kRitz][kRitz], V[kRitz][kRitz];
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
            A[i][j] = 0.5 * (S.T[i][j] + S.T[j][i]);
            V[i][j] = i == j ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < r; ++i) {
            diag += A[i][i] * A[i][i];
            for (int j = i + 1; j < r; ++j) off += A[i][j] * A[i][j];
        }
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < r; ++p)
            for (int q = p + 1; q < r; ++q) {
                if (A[p][q] == 0.0) continue;
                // rotation angle that zeroes A[p][q]: tan(phi) = t, the
                // smaller root of t^2 + 2 theta t - 1 = 0
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int i = 0; i < r; ++i) {  // columns p, q
                    const double aip = A[i][p], aiq = A[i][q];
                    A[i][p] = cs * aip - sn * aiq;
                    A[i][q] = sn * aip + cs * aiq;
                }
                for (int j = 0; j < r; ++j) {  // rows p, q
                    const double apj = A[p][j], aqj = A[q][j];
                    A[p][j] = cs * apj - sn * aqj;
                    A[q][j] = sn * apj + cs * aqj;
                }
                for (int i = 0; i < r; ++i) {
                    const double vip = V[i][p], viq = V[i][q];
                    V[i][p] = cs * vip - sn * viq;
                    V[i][q] = sn * vip + cs * viq;
                }
            }
    }
    int ord[kRitz];
    for (int i = 0; i < r; ++i) ord[i] = i;
    for (int i = 0; i < r; ++i)
        for (int j = i + 1; j < r; ++j)
            if (A[ord[j]][ord[j]] > A[ord[i]][ord[i]]) {
                const int x = ord[i];
                ord[i] = ord[j];
                ord[j] = x;
            }
    for (int c = 0; c < r; ++c) {
        S.lam[c] = A[ord[c]][ord[c]];
        for (int i = 0; i < r; ++i) S.U[i][c] = V[i][ord[c]];
    }
}

// M (k x k, global scratch) <- C^T C from G and s; then the two leading
// eigenvectors; then the layout coefficients w (2 x k) and offsets o.
__global__ void __launch_bounds__(kThreads) k_pmds_eig(const unsigned long long* __restrict__ G,
                                                       const unsigned long long* __restrict__ colsum, int32_t n,
                                                       int32_t k, double* __restrict__ M, double* __restrict__ W,
                                                       PmdsEig* __restrict__ out, StatusBlock* st)
{
    __shared__ EigSmem S;
    const int r = min(kRitz, k);
    const double invn = 1.0 / (double)n;
    // G' = G - s s^T / n
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += kThreads) {
        const int j = (int)(e / k), l = (int)(e % k);
        const size_t idx = (size_t)min(j, l) * k + max(j, l);
        const double g = (double)G[2 * idx + 1] * 0x1p64 + (double)G[2 * idx];
        M[e] = g - (double)colsum[j] * (double)colsum[l] * invn;
    }
    __syncthreads();
    // J_k G' J_k / 4 (G' is symmetric: its row and column means agree)
    for (int j = threadIdx.x; j < k; j += kThreads) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += M[(size_t)j * k + l];
        S.Z[j][0] = s / k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += S.Z[j][0];
        S.scal[0] = s / k;
    }
    __syncthreads();
    const double gm = S.scal[0];
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += kThreads) {
        const int j = (int)(e / k), l = (int)(e % k);
        M[e] = 0.25 * (M[e] - S.Z[j][0] - S.Z[l][0] + gm);
    }
    __syncthreads();

    for (int j = threadIdx.x; j < k; j += kThreads)
        for (int c = 0; c < r; ++c) S.Q[j][c] = start_value(j, c, 0);
    __syncthreads();
    orthonormalise(S, k, r, 1);
    double (*red16)[kRitz * kRitz] = S.red;
    double (*red2)[2] = reinterpret_cast<double (*)[2]>(&S.red[0][0]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int it = 0, converged = 0;
    for (; it < kEigMaxIter; ++it) {
        // Z = M Q: a warp per row, lanes over the row
        for (int j = warp; j < k; j += kThreads / 32) {
            double z[kRitz] = {0.0, 0.0, 0.0, 0.0};
            for (int l = lane; l < k; l += 32) {
                const double m = M[(size_t)j * k + l];
#pragma unroll
                for (int c = 0; c < kRitz; ++c)
                    if (c < r) z[c] += m * S.Q[l][c];
            }
#pragma unroll
            for (int c = 0; c < kRitz; ++c) z[c] = warp_sum(z[c]);
            if (lane == 0)
                for (int c = 0; c < r; ++c) S.Z[j][c] = z[c];
        }
        __syncthreads();
        // Rayleigh-Ritz: T = Q^T Z
        double tv[kRitz * kRitz];
#pragma unroll
        for (int i = 0; i < kRitz * kRitz; ++i) tv[i] = 0.0;
        for (int j = threadIdx.x; j < k; j += kThreads)
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) tv[a * kRitz + b] += S.Q[j][a] * S.Z[j][b];
        block_sums<kRitz * kRitz>(tv, red16);
        if (threadIdx.x == 0) {
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) S.T[a][b] = tv[a * kRitz + b];
            small_eigen(S, r);
        }
        __syncthreads();
        // Ritz vectors X = Q U (in Q) and M X = Z U (in Z)
        for (int j = threadIdx.x; j < k; j += kThreads) {
            double x[kRitz], y[kRitz];
            for (int c = 0; c < r; ++c) {
                x[c] = 0.0;
                y[c] = 0.0;
                for (int a = 0; a < r; ++a) {
                    x[c] += S.Q[j][a] * S.U[a][c];
                    y[c] += S.Z[j][a] * S.U[a][c];
                }
            }
            for (int c = 0; c < r; ++c) {
                S.Q[j][c] = x[c];
                S.Z[j][c] = y[c];
            }
        }
        __syncthreads();
        double res[2] = {0.0, 0.0};
        for (int j = threadIdx.x; j < k; j += kThreads)
            for (int c = 0; c < min(2, r); ++c) {
                const double e = S.Z[j][c] - S.lam[c] * S.Q[j][c];
                res[c] += e * e;
            }
        block_sums<2>(res, red2);
        const double bound = kEigTol * fabs(S.lam[0]);
        if (res[0] <= bound * bound && res[1] <= bound * bound) {
            converged = 1;
            break;
        }
        if (it + 1 == kEigMaxIter) break;
        for (int j = threadIdx.x; j < k; j += kThreads)
            for (int c = 0; c < r; ++c) S.Q[j][c] = S.Z[j][c];
        __syncthreads();
        orthonormalise(S, k, r, 2 + it);
    }
    // coefficients of the two axes
    for (int d = 0; d < 2; ++d) {
        const bool axis = d < r && S.lam[0] > 0.0 && S.lam[d] > kAxisEps * S.lam[0];
        // sign: the first entry (smallest index) whose magnitude is within a
        // relative kSignSlack of the largest is made positive
        double amax = 0.0;
        for (int j = threadIdx.x; j < k; j += kThreads) amax = fmax(amax, fabs(S.Q[j][d]));
        for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(FULL, amax, o));
        if (lane == 0) S.red[warp][0] = amax;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int q = 0; q < kThreads / 32; ++q) m = fmax(m, S.red[q][0]);
            S.scal[2] = m;
        }
        __syncthreads();
        const double thr = (1.0 - kSignSlack) * S.scal[2];
        int firstj = 0x7fffffff;
        for (int j = threadIdx.x; j < k; j += kThreads)
            if (fabs(S.Q[j][d]) >= thr) {
                firstj = j;
                break;
            }
        for (int o = 16; o > 0; o >>= 1) firstj = min(firstj, __shfl_xor_sync(FULL, firstj, o));
        if (lane == 0) S.red[warp][1] = (double)firstj;
        __syncthreads();
        if (threadIdx.x == 0) {
            int bj = 0x7fffffff;
            for (int q = 0; q < kThreads / 32; ++q) bj = min(bj, (int)S.red[q][1]);
            S.scal[1] = (bj < k && S.Q[bj][d] < 0.0) ? -1.0 : 1.0;
        }
        __syncthreads();
        const double sgn = S.scal[1];
        // J_k v: remove the mean over the pivots
        double mv[1] = {0.0};
        for (int j = threadIdx.x; j < k; j += kThreads) mv[0] += S.Q[j][d];
        block_sums<1>(mv, reinterpret_cast<double (*)[1]>(&S.red[0][0]));
        const double mean = mv[0] / k;
        const double scale = axis ? -0.5 * sgn / sqrt(sqrt(S.lam[d])) : 0.0;
        double ov[1] = {0.0};
        for (int j = threadIdx.x; j < k; j += kThreads) {
            const double w = scale * (S.Q[j][d] - mean);
            W[(size_t)d * k + j] = w;
            ov[0] += (double)colsum[j] * invn * w;
        }
        block_sums<1>(ov, reinterpret_cast<double (*)[1]>(&S.red[0][0]));
        if (threadIdx.x == 0) {
            out->o[d] = ov[0];
            out->lam[d] = d < r ? S.lam[d] : 0.0;
        }
    }
    if (threadIdx.x == 0) {
        out->iters = it + 1;
        out->converged = converged;
        if (!converged) atomicOr(&st->warn, LTSNET_WARN_NOT_CONVERGED);
    }
}

// ---------------------------------------------------------------------------
// Step 5: layout and scale.

__global__ void __launch_bounds__(kThreads) k_pmds_layout(const uint16_t* __restrict__ D, int32_t n, int32_t k,
                                                          const int32_t* __restrict__ dmax,
                                                          const double* __restrict__ W,
                                                          const PmdsEig* __restrict__ eig, double2* __restrict__ XY,
                                                          double* __restrict__ partial)
{
    __shared__ double w0[kMaxPivots], w1[kMaxPivots];
    __shared__ double red[kThreads / 32];
    for (int j = threadIdx.x; j < k; j += kThreads) {
        w0[j] = W[j];
        w1[j] = W[(size_t)k + j];
    }
    __syncthreads();
    const uint32_t fill = (uint32_t)*dmax + 1u;
    const double o0 = eig->o[0], o1 = eig->o[1];
    double ss = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int j = 0; j < k; ++j) {
            const double a = (double)sq_dist(D[(size_t)j * n + i], fill);
            x = fma(a, w0[j], x);
            y = fma(a, w1[j], y);
        }
        x -= o0;
        y -= o1;
        XY[i] = make_double2(x, y);
        ss += x * x + y * y;
    }
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) s += red[q];
        partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads) k_pmds_scale(const double2* __restrict__ XY, int32_t n,
                                                         const double* __restrict__ partial, int32_t nparts,
                                                         double init_std, float2* __restrict__ Y)
{
    __shared__ double f;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < nparts; ++q) s += partial[q];
        const double rms = sqrt(s / (2.0 * (double)n));
        f = (init_std > 0.0 && rms > 0.0) ? init_std / rms : 1.0;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = XY[i];
        Y[i] = make_float2((float)(v.x * f), (float)(v.y * f));
    }
}

struct PmdsWs {
    StatusBlock* st;
    LevelCtl* ctl;
    PmdsEig* eig;
    int32_t* dmax;
    uint16_t* D;
    int32_t* q0;
    int32_t* q1;
    uint32_t* nearest;
    unsigned long long* best;
    unsigned long long* colsum;
    unsigned long long* G;
    double* M;
    double* W;
    double2* XY;
    double* partial;
};

size_t pmds_carve(void* ws, int32_t n, int32_t k, PmdsWs* w)
{
    Carve c(ws, ~(size_t)0);
    PmdsWs t;
    t.st = c.take<StatusBlock>(1);
    t.ctl = c.take<LevelCtl>(1);
    t.eig = c.take<PmdsEig>(1);
    t.dmax = c.take<int32_t>(1);
    t.D = c.take<uint16_t>((size_t)k * n);
    t.q0 = c.take<int32_t>(n);
    t.q1 = c.take<int32_t>(n);
    t.nearest = c.take<uint32_t>(n);
    t.best = c.take<unsigned long long>(k);
    t.colsum = c.take<unsigned long long>(k);
    t.G = c.take<unsigned long long>((size_t)2 * k * k);
    t.M = c.take<double>((size_t)k * k);
    t.W = c.take<double>((size_t)2 * k);
    t.XY = c.take<double2>(n);
    t.partial = c.take<double>(kFlatBlocks);
    if (w) *w = t;
    return align_up(c.off, 256);
}

}  // namespace
}  // namespace lt

extern "C" size_t ltsnet_pivot_mds_workspace_size(int32_t n, int32_t n_pivots)
{
    if (n < 2 || n_pivots < 2 || n_pivots > lt::kMaxPivots || n_pivots > n) return 0;
    return lt::pmds_carve(nullptr, n, n_pivots, nullptr);
}

extern "C" ltsnet_status ltsnet_pivot_mds(const int64_t* row_ptr, const int32_t* col, int32_t n, int32_t n_pivots,
                                          int32_t first_pivot, double init_std, float* Y, int32_t* pivots,
                                          uint16_t* dist, double* eigvals, void* ws, size_t ws_bytes,
                                          ltsnet_stream stream)
{
    using namespace lt;
    const int32_t k = n_pivots;
    if (n < 2 || k < 2 || k > kMaxPivots || k > n || first_pivot < 0 || first_pivot >= n || !(init_std >= 0.0) ||
        !isfinite(init_std) || !row_ptr || !col || !Y || !pivots || !ws)
        return LTSNET_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255) || ws_bytes < pmds_carve(nullptr, n, k, nullptr)) return LTSNET_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    PmdsWs w;
    pmds_carve(ws, n, k, &w);
    uint16_t* D = dist ? dist : w.D;

    LT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StatusBlock), s));
    LT_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(LevelCtl), s));
    LT_CUDA(cudaMemsetAsync(w.dmax, 0, sizeof(int32_t), s));
    LT_CUDA(cudaMemsetAsync(D, 0xFF, sizeof(uint16_t) * (size_t)k * n, s));
    LT_CUDA(cudaMemsetAsync(w.nearest, 0xFF, sizeof(uint32_t) * (size_t)n, s));
    LT_CUDA(cudaMemsetAsync(w.best, 0, sizeof(unsigned long long) * (size_t)k, s));
    LT_CUDA(cudaMemsetAsync(w.colsum, 0, sizeof(unsigned long long) * (size_t)k, s));
    LT_CUDA(cudaMemsetAsync(w.G, 0, sizeof(unsigned long long) * 2 * (size_t)k * k, s));

    LevelRunner lr{row_ptr, col, n, D, w.q0, w.q1, w.ctl, w.st};
    if (ltsnet_status e = lr.prepare()) return e;
    for (int32_t t = 0; t < k; ++t) {
        k_pmds_pivot<<<1, 1, 0, s>>>(t, first_pivot, n, w.best, pivots, D, w.q0, w.ctl, w.st);
        count_launches(1);
        LT_CHECK_LAUNCH();
        LevelCtl h;
        if (ltsnet_status e = lr.run(s, &h)) return e;
        if (h.err) break;
        k_pmds_nearest<<<kFlatBlocks, kThreads, 0, s>>>(D, t, n, w.nearest, t + 1 < k ? w.best + t + 1 : nullptr,
                                                         w.dmax);
        count_launches(1);
        LT_CHECK_LAUNCH();
    }
    StatusBlock hs;
    LT_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    if (hs.code) return (ltsnet_status)hs.code;

    const int nsplit = std::max(1, std::min(kFlatBlocks, (int)((n + 4095) / 4096)));
    k_pmds_colsum<<<dim3(nsplit, k), kThreads, 0, s>>>(D, n, w.dmax, w.colsum);
    count_launches(1);
    LT_CHECK_LAUNCH();
    const int ntb = (k + kTile - 1) / kTile;
    const int ntiles = ntb * (ntb + 1) / 2;
    int splits = std::max(1, (num_sms() * 4 + ntiles - 1) / ntiles);
    int64_t rows = ((int64_t)n + splits - 1) / splits;
    rows = (rows + kRows - 1) / kRows * kRows;
    splits = (int)(((int64_t)n + rows - 1) / rows);
    k_pmds_gram<<<dim3(ntiles, splits), kThreads, 0, s>>>(D, n, k, (int32_t)rows, w.dmax, w.G);
    count_launches(1);
    LT_CHECK_LAUNCH();
    k_pmds_eig<<<1, kThreads, 0, s>>>(w.G, w.colsum, n, k, w.M, w.W, w.eig, w.st);
    count_launches(1);
    LT_CHECK_LAUNCH();
    k_pmds_layout<<<kFlatBlocks, kThreads, 0, s>>>(D, n, k, w.dmax, w.W, w.eig, w.XY, w.partial);
    count_launches(1);
    LT_CHECK_LAUNCH();
    k_pmds_scale<<<kFlatBlocks, kThreads, 0, s>>>(w.XY, n, w.partial, kFlatBlocks, init_std, (float2*)Y);
    count_launches(1);
    LT_CHECK_LAUNCH();
    PmdsEig he;
    LT_CUDA(cudaMemcpyAsync(&he, w.eig, sizeof(PmdsEig), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    if (eigvals) {
        eigvals[0] = he.lam[0];
        eigvals[1] = he.lam[1];
    }
    if (hs.code) return (ltsnet_status)hs.code;
    return hs.warn ? LTSNET_WARN_NOT_CONVERGED : LTSNET_OK;
}
