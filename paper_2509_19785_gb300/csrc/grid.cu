// Interpolation grid of one iteration (Sec. 2.3 "four sums", Sec. 3.3 h1..h3,
// Alg. 3 loop): grid rule, spreading, FFT convolution with the kernels
// (1+d^2)^-2 and 1/(eps+d^2), and Z.
//
// The sums are those of the paper's interpolation (FIt-SNE's "four sums" and
// the L-tsNET entropy sums h1, h2, h3), rearranged exactly so that FP32 loses
// nothing to cancellation.  With node positions xi, node spacing s and
// x_i - x_j = (x_i - xi_a) + (xi_a - xi_b) + (xi_b - x_j) for target node a
// and source node b, the repulsion sum becomes
//   R_x(i) = s sum_a L_a(i) [ e_x(i,a) (K2*S0)_a + ((K2 dx)*S0 - K2*S1x)_a ]
// with node-local charges S0 = sum L, S1 = sum L e, S2 = sum L |e|^2 (e the
// offset of a point from a node, in node spacings) and integer node offsets
// dx.  The same with Ke gives the entropy sum, and Z becomes a sum of
// products of these grids (evaluated by Parseval).  No term carries the
// layout's absolute coordinates, so the extent does not cost precision.
//
//  k_setup        grid rule from the layout bounds (FP32, same decisions as
//                 the oracle), FFT plan and twiddles, fixed-point scales.
//  k_bin_count    points -> spread tiles (48x48 nodes), counts per tile.
//  k_bin_plan     tile offsets and work items (tile, point range).
//  k_bin_scatter  points copied into their tile's range.
//  k_spread_tiles per work item: Lagrange weights x charges accumulated in a
//                 shared-memory tile as 64-bit fixed point (integer sums are
//                 order independent, so the grid is bit-identical from run to
//                 run), then flushed to the global fixed-point grid.
//  k_spread_atomic  the plain form: FP32 atomics straight into the grid.
//  k_spec_rows/cols 2-D FFTs of the kernels (K2, Ke, K1 even; K2 dx, Ke dx
//                 odd), three packed complex transforms, half spectra kept.
//  k_conv_rows_fwd  row FFTs of the charges, two real rows per complex line.
//  k_conv_cols    column FFTs, kernel products, inverse column FFTs, Z.
//  k_conv_rows_inv  inverse row FFTs, two real fields per complex line.
// Zero padding to L = 2M makes the circular convolution equal the linear one
// on the M x M node grid; all grids are real, so half spectra suffice.
#include <math.h>

#include "iter.cuh"

namespace lt {
namespace {

__device__ __forceinline__ bool smooth5(int v)
{
    if (v < 1) return false;
    while (v % 2 == 0) v /= 2;
    while (v % 3 == 0) v /= 3;
    while (v % 5 == 0) v /= 5;
    return v == 1;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// Forward DFT (e^{-2 pi i jk/L}) of `nl` lines of length L (stride ld) held in
// shared memory, mixed radix 4/2/3/5 Stockham autosort with ping-pong buffers
// a, b.  Returns the buffer holding the result.  All threads of the block
// must call it.
__device__ float2* fft_lines(float2* a, float2* b, int nl, int ld, const GridDev& g, const float2* tw)
{
    const int L = g.L;
    int Ns = 1;
    for (int st = 0; st < g.nst; ++st) {
        const int R = g.radix[st];
        const int nbf = L / R;
        const int ts = L / (Ns * R);
        const int wR = L / R;
        for (int idx = threadIdx.x; idx < nl * nbf; idx += blockDim.x) {
            const int line = idx / nbf;
            const int j = idx - line * nbf;
            const float2* in = a + line * ld;
            float2* out = b + line * ld;
            const int jm = j % Ns;
            const int ob = (j - jm) * R + jm;
            float2 v[5];
            v[0] = in[j];
            for (int r = 1; r < R; ++r) v[r] = cmul(in[j + r * nbf], tw[jm * r * ts]);
            if (R == 4) {
                const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
                const float2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
                out[ob] = cadd(t0, t2);
                out[ob + Ns] = make_float2(t1.x + t3.y, t1.y - t3.x);
                out[ob + 2 * Ns] = csub(t0, t2);
                out[ob + 3 * Ns] = make_float2(t1.x - t3.y, t1.y + t3.x);
            } else if (R == 2) {
                out[ob] = cadd(v[0], v[1]);
                out[ob + Ns] = csub(v[0], v[1]);
            } else {
                for (int q = 0; q < R; ++q) {
                    float2 acc = v[0];
                    for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], tw[((r * q) % R) * wR]));
                    out[ob + q * Ns] = acc;
                }
            }
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

__device__ void compute_grid(const int32_t* bounds, float bwm, int min_boxes, int max_boxes, int P, int32_t n,
                             GridDev& g)
{
    const float lo = ord2f(bounds[0]);
    const float hi = ord2f(bounds[1]);
    float ext = __fsub_rn(hi, lo);
    if (!(ext >= 1e-6f)) ext = 1e-6f;
    const float q = __fdiv_rn(ext, bwm);
    int I;
    if (!(q < (float)max_boxes)) I = max_boxes;
    else I = (int)ceilf(q);
    if (I < min_boxes) I = min_boxes;
    while (!smooth5(I)) ++I;
    if (I > max_boxes) {
        I = max_boxes;
        while (I > 1 && !smooth5(I)) --I;
    }
    g.lo = lo;
    g.hi = hi;
    g.ext = ext;
    g.h = __fdiv_rn(ext, (float)I);
    g.s = __fdiv_rn(g.h, (float)P);
    g.c = __fmul_rn(0.5f, __fadd_rn(lo, hi));
    g.I = I;
    g.P = P;
    g.M = I * P;
    g.L = 2 * g.M;
    // Spread tiles of tb x tb boxes: about kSpreadChunk points per tile at the
    // mean density, at most kMaxTiles tiles per dimension, at most 8 boxes
    // per dimension unless the tile count forces more.
    {
        const double per_box = (double)n / ((double)I * (double)I);
        int tb = (int)floor(sqrt((double)kSpreadChunk / (per_box > 1e-9 ? per_box : 1e-9)));
        tb = tb < 1 ? 1 : (tb > 8 ? 8 : tb);
        const int tmin = (I + kMaxTiles - 1) / kMaxTiles;
        g.tb = tb < tmin ? tmin : tb;
    }
    g.tiles = (I + g.tb - 1) / g.tb;
    int r = g.L, k = 0;
    while (r % 4 == 0) { g.radix[k++] = 4; r /= 4; }
    while (r % 2 == 0) { g.radix[k++] = 2; r /= 2; }
    while (r % 3 == 0) { g.radix[k++] = 3; r /= 3; }
    while (r % 5 == 0) { g.radix[k++] = 5; r /= 5; }
    g.nst = k;
    // node-local charges (1, ex, ey, ex^2 + ey^2) with |e| <= P in node units,
    // Lagrange weight products <= 8 for P <= 5
    const double qb[4] = {1.0, (double)P, (double)P, 2.0 * P * P};
    for (int c = 0; c < 4; ++c) {
        int ex;
        frexp((double)n * 8.0 * qb[c], &ex);
        g.fx[c] = ldexp(1.0, 62 - ex);
        g.ifx[c] = ldexp(1.0, ex - 62);
    }
}

__global__ void k_setup(const int32_t* __restrict__ bounds_cur, int32_t* __restrict__ bounds_next, GridDev* G,
                        float2* __restrict__ tw, int32_t* __restrict__ tile_cnt, int32_t n, float bwm, int min_boxes,
                        int max_boxes, int P)
{
    __shared__ GridDev g;
    if (threadIdx.x == 0) compute_grid(bounds_cur, bwm, min_boxes, max_boxes, P, n, g);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        G->lo = g.lo; G->hi = g.hi; G->ext = g.ext; G->h = g.h; G->s = g.s; G->c = g.c;
        G->I = g.I; G->M = g.M; G->L = g.L; G->P = g.P; G->tb = g.tb; G->tiles = g.tiles;
        G->nst = g.nst;
        for (int i = 0; i < kMaxRadix; ++i) G->radix[i] = i < g.nst ? g.radix[i] : 0;
        for (int c = 0; c < 4; ++c) { G->fx[c] = g.fx[c]; G->ifx[c] = g.ifx[c]; }
        G->ticket = 0;
        G->nitems = 0;
        bounds_next[0] = f2ord(INFINITY);
        bounds_next[1] = f2ord(-INFINITY);
    }
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = tid; t < g.L; t += nth) {
        // e^{-2 pi i t/L} = (-i)^q e^{-(pi/2) i r/L} with 4t = q L + r, 0 <= r < L:
        // the reduced argument r/L is in [0, 1) and correctly rounded.
        const int q = (int)((4 * t) / g.L), r = (int)(4 * t - (int64_t)q * g.L);
        float sn, cs;
        sincospif(-0.5f * ((float)r / (float)g.L), &sn, &cs);
        float2 v;
        if (q == 0) v = make_float2(cs, sn);
        else if (q == 1) v = make_float2(sn, -cs);
        else if (q == 2) v = make_float2(-cs, -sn);
        else v = make_float2(-sn, cs);
        tw[t] = v;
    }
    for (int64_t t = tid; t < (int64_t)g.tiles * g.tiles; t += nth) tile_cnt[t] = 0;
}

__global__ void k_bin_count(const float2* __restrict__ Y, int32_t n, const GridDev* __restrict__ G,
                            int32_t* __restrict__ tile_cnt)
{
    extern __shared__ int32_t sh[];
    const float lo = G->lo, h = G->h;
    const int I = G->I, tb = G->tb, tiles = G->tiles, T = tiles * tiles;
    for (int t = threadIdx.x; t < T; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = Y[i];
        const int bx = box_of(p.x, lo, h, I), by = box_of(p.y, lo, h, I);
        atomicAdd(&sh[(by / tb) * tiles + bx / tb], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        if (sh[t]) atomicAdd(&tile_cnt[t], sh[t]);
}

// Single block: exclusive scan of the tile counts and the work-item list.
__global__ void k_bin_plan(GridDev* G, const int32_t* __restrict__ tile_cnt, int32_t* __restrict__ tile_off,
                           int32_t* __restrict__ tile_cur, int4* __restrict__ items, int32_t chunk)
{
    __shared__ int32_t wsum[33];
    __shared__ int32_t carry_pts, carry_items;
    const int T = G->tiles * G->tiles;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        carry_pts = 0;
        carry_items = 0;
    }
    __syncthreads();
    for (int t0 = 0; t0 < T; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const int c = t < T ? tile_cnt[t] : 0;
        const int ni = (c + chunk - 1) / chunk;
        int vals[2] = {c, ni};
        int excl[2], tot[2];
        for (int k = 0; k < 2; ++k) {
            int inc = vals[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += u;
            }
            if (lane == 31) wsum[w] = inc;
            __syncthreads();
            if (w == 0) {
                int x = lane < nw ? wsum[lane] : 0, xi = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int u = __shfl_up_sync(FULL, xi, o);
                    if (lane >= o) xi += u;
                }
                if (lane < nw) wsum[lane] = xi - x;
                if (lane == 31) wsum[32] = xi;
            }
            __syncthreads();
            excl[k] = wsum[w] + inc - vals[k];
            tot[k] = wsum[32];
            __syncthreads();
        }
        if (t < T) {
            const int off = carry_pts + excl[0];
            tile_off[t] = off;
            tile_cur[t] = off;
            const int ib = carry_items + excl[1];
            for (int q = 0; q < ni; ++q) {
                const int b = off + q * chunk;
                const int e = min(off + c, b + chunk);
                items[ib + q] = make_int4(t, b, e, ni == 1 ? 1 : 0);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_pts += tot[0];
            carry_items += tot[1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tile_off[T] = carry_pts;
        G->nitems = carry_items;
    }
}

__global__ void k_bin_scatter(const float2* __restrict__ Y, int32_t n, const GridDev* __restrict__ G,
                              int32_t* __restrict__ tile_cur, float2* __restrict__ binned)
{
    extern __shared__ int32_t sh[];
    const float lo = G->lo, h = G->h;
    const int I = G->I, tb = G->tb, tiles = G->tiles, T = tiles * tiles;
    int32_t* cnt = sh;
    int32_t* base = sh + T;
    constexpr int kItems = 8;
    for (int t = threadIdx.x; t < T; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * blockDim.x * kItems;
    int tl[kItems], rk[kItems];
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t i = b0 + (int64_t)q * blockDim.x + threadIdx.x;
        tl[q] = -1;
        rk[q] = 0;
        if (i < n) {
            const float2 p = Y[i];
            const int bx = box_of(p.x, lo, h, I), by = box_of(p.y, lo, h, I);
            tl[q] = (by / tb) * tiles + bx / tb;
            rk[q] = atomicAdd(&cnt[tl[q]], 1);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        base[t] = cnt[t] ? atomicAdd(&tile_cur[t], cnt[t]) : 0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t i = b0 + (int64_t)q * blockDim.x + threadIdx.x;
        if (tl[q] >= 0) binned[base[tl[q]] + rk[q]] = Y[i];
    }
}

// One work item = one tile of tb x tb boxes and up to kSpreadChunk of its
// points (tiles are sized for about one item at the mean density).  The
// points are counting-sorted by box in shared memory, their local
// coordinates computed once on the way.  Each thread then takes one node row
// of a contiguous slice of the sorted points and accumulates that row's P
// nodes x 4 charges in 64-bit fixed point in registers, adding them into a
// shared-memory tile when the box changes; the tile is stored to the global
// fixed-point grid (added atomically when a dense tile has several items).
// Integer sums do not depend on order, so the grid is the same bit for bit
// from run to run.
template <int P>
__global__ void __launch_bounds__(256) k_spread_tiles(const float2* __restrict__ binned, const GridDev* __restrict__ G,
                                                      const int4* __restrict__ items, long long* __restrict__ wfix)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = G->M, I = G->I, tb = G->tb, tiles = G->tiles;
    const float lo = G->lo, h = G->h, s = G->s;
    const int NB = tb * tb, TN = tb * P;
    long long* acc = (long long*)smraw;                      // TN * TN * 4
    float2* su = (float2*)(acc + kMaxTileNodes * kMaxTileNodes * 4);  // kSpreadChunk
    int* slb = (int*)(su + kSpreadChunk);                    // kSpreadChunk
    int* off = slb + kSpreadChunk;                           // NB + 1
    int* cur = off + kMaxTileBoxes + 1;                      // NB
    float fx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) fx[q] = (float)G->fx[q];
    const int nslice = blockDim.x / P;
    const int nitems = G->nitems;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 item = items[it];
        const int tx = item.x % tiles, ty = item.x / tiles;
        const int bx0 = tx * tb, by0 = ty * tb;
        const int cnt = item.z - item.y;
        for (int i = threadIdx.x; i < TN * TN * 4; i += blockDim.x) acc[i] = 0;
        for (int i = threadIdx.x; i < NB; i += blockDim.x) cur[i] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            const float2 p = binned[item.y + j];
            const int lb = (box_of(p.y, lo, h, I) - by0) * tb + (box_of(p.x, lo, h, I) - bx0);
            atomicAdd(&cur[lb], 1);
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // exclusive scan of the box counts by warp 0
            int carry = 0;
            for (int b0 = 0; b0 < NB; b0 += 32) {
                const int b = b0 + threadIdx.x;
                const int v = b < NB ? cur[b] : 0;
                int inc = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(FULL, inc, o);
                    if (threadIdx.x >= o) inc += t;
                }
                if (b < NB) {
                    off[b] = carry + inc - v;
                    cur[b] = carry + inc - v;
                }
                carry += __shfl_sync(FULL, inc, 31);
            }
            if (threadIdx.x == 0) off[NB] = carry;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            const float2 p = binned[item.y + j];
            const int bx = box_of(p.x, lo, h, I), by = box_of(p.y, lo, h, I);
            const int lb = (by - by0) * tb + (bx - bx0);
            const int pos = atomicAdd(&cur[lb], 1);
            su[pos] = make_float2(local_u(p.x, lo, s, P * bx), local_u(p.y, lo, s, P * by));
            slb[pos] = lb;
        }
        __syncthreads();
        if (threadIdx.x < nslice * P) {
            const int slice = threadIdx.x / P, bb = threadIdx.x - slice * P;
            const int per = (cnt + nslice - 1) / nslice;
            const int q0 = slice * per, q1 = min(cnt, q0 + per);
            long long ra[P][4];
            int cur_lb = -1;
            for (int q = q0; q <= q1; ++q) {
                const int lb = q < q1 ? slb[q] : -2;
                if (lb != cur_lb) {
                    if (cur_lb >= 0) {
                        const int ly = (cur_lb / tb) * P + bb, lx0 = (cur_lb % tb) * P;
                        long long* dst = acc + (ly * TN + lx0) * 4;
#pragma unroll
                        for (int a = 0; a < P; ++a)
#pragma unroll
                            for (int ch = 0; ch < 4; ++ch)
                                if (ra[a][ch] != 0)
                                    atomicAdd((unsigned long long*)(dst + a * 4 + ch), (unsigned long long)ra[a][ch]);
                    }
                    if (q == q1) break;
                    cur_lb = lb;
#pragma unroll
                    for (int a = 0; a < P; ++a)
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) ra[a][ch] = 0;
                }
                const float2 u = su[q];
                float wx[P];
                lagrange<P>(u.x, wx);
                const float wyb = lagrange_one<P>(u.y, bb);
                const float ey = u.y - ((float)bb + 0.5f);
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const float w = wx[a] * wyb;
                    const float ex = u.x - ((float)a + 0.5f);
                    ra[a][0] += __float2ll_rn(w * fx[0]);
                    ra[a][1] += __float2ll_rn((w * ex) * fx[1]);
                    ra[a][2] += __float2ll_rn((w * ey) * fx[2]);
                    ra[a][3] += __float2ll_rn((w * (ex * ex + ey * ey)) * fx[3]);
                }
            }
        }
        __syncthreads();
        const bool single = item.w != 0;
        for (int i = threadIdx.x; i < TN * TN * 4; i += blockDim.x) {
            const long long v = acc[i];
            if (v == 0) continue;
            const int node = i >> 2, ch = i & 3;
            const int gy = by0 * P + node / TN, gx = bx0 * P + node % TN;
            if (gy >= M || gx >= M) continue;
            long long* dst = wfix + ((int64_t)gy * M + gx) * 4 + ch;
            if (single) *dst = v;
            else atomicAdd((unsigned long long*)dst, (unsigned long long)v);
        }
        __syncthreads();
    }
}

template <int P>
__global__ void k_spread_atomic(const float2* __restrict__ Y, int32_t n, const GridDev* __restrict__ G,
                                float4* __restrict__ wflt)
{
    const int M = G->M;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int bx, by;
        float ux, uy;
        local_coords(Y[i], G, bx, by, ux, uy);
        float wx[P], wy[P];
        lagrange<P>(ux, wx);
        lagrange<P>(uy, wy);
#pragma unroll
        for (int b = 0; b < P; ++b)
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const float w = wx[a] * wy[b];
                const float ex = ux - ((float)a + 0.5f), ey = uy - ((float)b + 0.5f);
                atomicAdd(wflt + (int64_t)(P * by + b) * M + (P * bx + a),
                          make_float4(w, w * ex, w * ey, w * (ex * ex + ey * ey)));
            }
    }
}

// Work split: block b takes units [b*per, min(total, (b+1)*per)).
__device__ __forceinline__ void block_range(int total, int& beg, int& end)
{
    const int per = (total + gridDim.x - 1) / gridDim.x;
    beg = blockIdx.x * per;
    end = min(total, beg + per);
}

__device__ __forceinline__ void load_tw(float2* stw, const float2* __restrict__ tw, int L)
{
    for (int t = threadIdx.x; t < L; t += blockDim.x) stw[t] = tw[t];
}

// Lines of length L that fit `bufs` buffers next to the twiddles.
__device__ __forceinline__ int line_cap(int sm_f2, int L, int bufs)
{
    const int c = (sm_f2 - L) / (bufs * L);
    return c < 1 ? 1 : c;
}

// Signed node offset of circulant index a in [0, L): a for a < M, a - L for
// a > L - M, none (the unused middle index) otherwise.
__device__ __forceinline__ bool circ_offset(int a, int M, int L, int& d)
{
    if (a < M) { d = a; return true; }
    if (a > L - M) { d = a - L; return true; }
    return false;
}

constexpr float kEntScale = 0.125f;  // Ke is packed scaled by 1/8 to match K2's magnitude

// Kernel spectra, pass 1: rows a in [0, L) of the circulant embeddings of
// three packed complex kernels over node offsets (dx, dy), d^2 = s^2 |.|^2:
//   q = 0: K2 + i Ke/8      q = 1: K1      q = 2: K2 dx + i Ke dx / 8
// transformed along x; columns kx in [0, L/2] are kept (all five kernels are
// even or odd in x, so the other half follows by symmetry).
__global__ void k_spec_rows(const GridDev* __restrict__ Gp, const float2* __restrict__ tw, float eps,
                            float2* __restrict__ krow, int sm_f2)
{
    extern __shared__ float2 smf[];
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    const float s2 = G.s * G.s;
    const int cap = line_cap(sm_f2, L, 2);
    float2* stw = smf;
    float2* A = smf + L;
    float2* B = A + (size_t)cap * L;
    load_tw(stw, tw, L);
    int beg, end;
    block_range(3 * L, beg, end);  // unit = (q, a)
    for (int u0 = beg; u0 < end; u0 += cap) {
        const int nl = min(cap, end - u0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
            const int line = idx / L, b = idx - line * L;
            const int u = u0 + line, q = u / L, a = u - q * L;
            int dx, dy;
            float2 v = make_float2(0.f, 0.f);
            if (circ_offset(b, M, L, dx) && circ_offset(a, M, L, dy)) {
                const float d2 = s2 * (float)(dx * dx + dy * dy);
                const float k1 = 1.0f / (1.0f + d2);
                const float ke = kEntScale / (eps + d2);
                if (q == 0) v = make_float2(k1 * k1, ke);
                else if (q == 1) v = make_float2(k1, 0.f);
                else v = make_float2(k1 * k1 * (float)dx, ke * (float)dx);
            }
            A[line * L + b] = v;
        }
        __syncthreads();
        float2* R = fft_lines(A, B, nl, L, G, stw);
        for (int idx = threadIdx.x; idx < nl * H; idx += blockDim.x) {
            const int line = idx / H, k = idx - line * H;
            const int u = u0 + line, q = u / L, a = u - q * L;
            krow[((int64_t)q * L + a) * H + k] = R[line * L + k];
        }
    }
}

// Kernel spectra, pass 2: columns kx in [0, L/2], scaled by 1/L^2 (the inverse
// transforms are unnormalised).  khat[f][ky][kx], f = 0: K2^, 1: Ke^, 2: K1^
// (real), 3: Im (K2 dx)^, 4: Im (Ke dx)^ (those two spectra are imaginary).
__global__ void k_spec_cols(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                            const float2* __restrict__ krow, float* __restrict__ khat, int sm_f2)
{
    extern __shared__ float2 smf[];
    const GridDev& G = *Gp;
    const int L = G.L, H = L / 2 + 1;
    const float scale = 1.0f / ((float)L * (float)L);
    const int cap = line_cap(sm_f2, L, 2);
    float2* stw = smf;
    float2* A = smf + L;
    float2* B = A + (size_t)cap * L;
    load_tw(stw, tw, L);
    const int64_t LH = (int64_t)L * H;
    int beg, end;
    block_range(3 * H, beg, end);  // unit = (q, kx)
    for (int u0 = beg; u0 < end; u0 += cap) {
        const int nl = min(cap, end - u0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
            const int a = idx / nl, line = idx - a * nl;
            const int u = u0 + line, q = u / H, kx = u - q * H;
            A[line * L + a] = krow[(int64_t)q * LH + (int64_t)a * H + kx];
        }
        __syncthreads();
        float2* R = fft_lines(A, B, nl, L, G, stw);
        for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
            const int ky = idx / nl, line = idx - ky * nl;
            const int u = u0 + line, q = u / H, kx = u - q * H;
            const float2 v = R[line * L + ky];
            const int64_t o = (int64_t)ky * H + kx;
            if (q == 0) {
                khat[0 * LH + o] = v.x * scale;
                khat[1 * LH + o] = v.y * scale / kEntScale;
            } else if (q == 1) {
                khat[2 * LH + o] = v.x * scale;
            } else {
                // FFT(K2dx + i Ke dx/8) = i b2 + i (i be/8) = -be/8 + i b2
                khat[3 * LH + o] = v.y * scale;
                khat[4 * LH + o] = -v.x * scale / kEntScale;
            }
        }
    }
}

__device__ __forceinline__ float4 load_charges(const long long* __restrict__ wfix, const float4* __restrict__ wflt,
                                               int plain, const GridDev& G, int64_t node)
{
    if (plain) return wflt[node];
    const long long* p = wfix + node * 4;
    return make_float4((float)((double)p[0] * G.ifx[0]), (float)((double)p[1] * G.ifx[1]),
                       (float)((double)p[2] * G.ifx[2]), (float)((double)p[3] * G.ifx[3]));
}

// Row FFTs of the charge grids S0, S1x, S1y, S2 (node-local moments), packed
// two real rows per complex line (S0 + i S1x, S1y + i S2) and separated by
// Hermitian symmetry into half spectra srow[g][ty][kx], kx in [0, L/2].
__global__ void k_conv_rows_fwd(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                                const long long* __restrict__ wfix, const float4* __restrict__ wflt, int plain,
                                float2* __restrict__ srow, int sm_f2)
{
    extern __shared__ float2 smf[];
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    const int cap = line_cap(sm_f2, L, 2);
    float2* stw = smf;
    float2* A = smf + L;
    float2* B = A + (size_t)cap * L;
    load_tw(stw, tw, L);
    const int64_t MH = (int64_t)M * H;
    int beg, end;
    block_range(2 * M, beg, end);  // unit = (pair, row): pair 0 = (S0, S1x), 1 = (S1y, S2)
    for (int u0 = beg; u0 < end; u0 += cap) {
        const int nl = min(cap, end - u0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
            const int line = idx / L, x = idx - line * L;
            const int u = u0 + line, pr = u / M, row = u - pr * M;
            float2 v = make_float2(0.f, 0.f);
            if (x < M) {
                const float4 w = load_charges(wfix, wflt, plain, G, (int64_t)row * M + x);
                v = pr == 0 ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
            }
            A[line * L + x] = v;
        }
        __syncthreads();
        float2* R = fft_lines(A, B, nl, L, G, stw);
        for (int idx = threadIdx.x; idx < nl * H; idx += blockDim.x) {
            const int line = idx / H, k = idx - line * H;
            const int u = u0 + line, pr = u / M, row = u - pr * M;
            const float2 z = R[line * L + k];
            const float2 zc = conj2(R[line * L + (k == 0 ? 0 : L - k)]);
            const float2 re = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y + zc.y));
            const float2 df = make_float2(z.x - zc.x, z.y - zc.y);
            const float2 im = make_float2(0.5f * df.y, -0.5f * df.x);  // (z - zc) / 2i
            srow[(int64_t)(2 * pr) * MH + (int64_t)row * H + k] = re;
            srow[(int64_t)(2 * pr + 1) * MH + (int64_t)row * H + k] = im;
        }
    }
}

// Column pass, kx in [0, L/2]: FFT along y of the four charge spectra, the
// products with the kernel spectra (node-local form of the repulsion and
// entropy sums), inverse FFTs along y (conjugation trick), rows < M kept:
//   U0 = K2^ S0^                 (F0)
//   U1 = Ke^ S0^                 (Fe0)
//   U2 = (K2 dx)^ S0^ - K2^ S1x^ (Vx)     U3 = (K2 dy)^ S0^ - K2^ S1y^ (Vy)
//   U4 = (Ke dx)^ S0^ - Ke^ S1x^ (Vex)    U5 = (Ke dy)^ S0^ - Ke^ S1y^ (Vey)
// and, by Parseval over the half spectrum, the grid sum
//   Z + n = sum [S0 (K1*S0) + 2 s^2 (S1 . (2 (K2 d)*S0 - K2*S1) + S2 (K2*S0))],
// accumulated in FP64 and finished by the last block in a fixed order.
__device__ __forceinline__ float odd_transposed(const float* __restrict__ Dh, int kx, int ky, int L, int H)
{
    // (K dy)^(kx, ky) = (K dx)^(ky, kx); stored half spectrum covers kx <= L/2,
    // the rest by oddness in the first argument.
    return ky <= L / 2 ? Dh[(int64_t)kx * H + ky] : -Dh[(int64_t)kx * H + (L - ky)];
}

// Z integrand at (kx, ky) from the four charge spectra (see k_conv_cols).
__device__ __forceinline__ double z_term(float2 s0, float2 s1x, float2 s1y, float2 s2v, float k2, float k1, float d2x,
                                         float d2y, float s2)
{
    const double gx_re = -2.0 * d2x * s0.y - k2 * s1x.x, gx_im = 2.0 * d2x * s0.x - k2 * s1x.y;
    const double gy_re = -2.0 * d2y * s0.y - k2 * s1y.x, gy_im = 2.0 * d2y * s0.x - k2 * s1y.y;
    double t = (double)k1 * ((double)s0.x * s0.x + (double)s0.y * s0.y);
    const double c = (double)s1x.x * gx_re + (double)s1x.y * gx_im + (double)s1y.x * gy_re + (double)s1y.y * gy_im +
                     (double)k2 * ((double)s2v.x * s0.x + (double)s2v.y * s0.y);
    return t + 2.0 * (double)s2 * c;
}

// Product q at (kx, ky) for the inverse column transform (conjugated).
__device__ __forceinline__ float2 conv_product(int q, float2 s0, float2 s1x, float2 s1y, const float* __restrict__ K2h,
                                               const float* __restrict__ Keh, const float* __restrict__ D2h,
                                               const float* __restrict__ Deh, int kx, int ky, int L, int H)
{
    const int64_t o = (int64_t)ky * H + kx;
    float2 v;
    if (q == 0) {
        const float k = K2h[o];
        v = make_float2(k * s0.x, k * s0.y);
    } else if (q == 1) {
        const float k = Keh[o];
        v = make_float2(k * s0.x, k * s0.y);
    } else {
        const bool ent = q >= 4;
        const bool ydir = (q & 1) != 0;
        const float* Dh = ent ? Deh : D2h;
        const float k = ent ? Keh[o] : K2h[o];
        const float d = ydir ? odd_transposed(Dh, kx, ky, L, H) : Dh[o];
        const float2 s1 = ydir ? s1y : s1x;
        v = make_float2(-d * s0.y - k * s1.x, d * s0.x - k * s1.y);
    }
    return conj2(v);
}

__global__ void k_conv_cols(GridDev* Gp, const float2* __restrict__ tw, const float2* __restrict__ srow,
                            const float* __restrict__ khat, float2* __restrict__ ucol, double* __restrict__ zblk,
                            int32_t n, int sm_f2)
{
    extern __shared__ float2 smf[];
    __shared__ double red[256];
    __shared__ bool last;
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    const float s2 = G.s * G.s;
    float2* stw = smf;
    load_tw(stw, tw, L);
    const int64_t MH = (int64_t)M * H, LH = (int64_t)L * H;
    const float* K2h = khat;
    const float* Keh = khat + LH;
    const float* K1h = khat + 2 * LH;
    const float* D2h = khat + 3 * LH;
    const float* Deh = khat + 4 * LH;
    double zacc = 0.0;
    int beg, end;
    block_range(H, beg, end);
    // Batched: 4 spectra + 6 products + 6 work lines per column, two FFT calls.
    const int capb = (sm_f2 - L) / (16 * L);
    if (capb >= 1) {
        for (int k0 = beg; k0 < end; k0 += capb) {
            const int nc = min(capb, end - k0);
            float2* SP = smf + L;
            float2* PR = SP + (size_t)4 * nc * L;
            float2* PP = PR + (size_t)6 * nc * L;
            __syncthreads();
            for (int idx = threadIdx.x; idx < 4 * nc * L; idx += blockDim.x) {
                const int y = idx / (4 * nc), r = idx - y * (4 * nc);
                const int gsel = r / nc, c = r - gsel * nc;
                SP[r * L + y] = y < M ? srow[(int64_t)gsel * MH + (int64_t)y * H + k0 + c] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            float2* R = fft_lines(SP, PP, 4 * nc, L, G, stw);
            if (R != SP) {
                for (int idx = threadIdx.x; idx < 4 * nc * L; idx += blockDim.x) SP[idx] = R[idx];
                __syncthreads();
            }
            for (int idx = threadIdx.x; idx < nc * L; idx += blockDim.x) {
                const int ky = idx / nc, c = idx - ky * nc;
                const int kx = k0 + c;
                const int64_t o = (int64_t)ky * H + kx;
                const float2 s0 = SP[(0 * nc + c) * L + ky], s1x = SP[(1 * nc + c) * L + ky];
                const float2 s1y = SP[(2 * nc + c) * L + ky], s2v = SP[(3 * nc + c) * L + ky];
                const double wgt = (kx == 0 || 2 * kx == L) ? 1.0 : 2.0;
                zacc += wgt * z_term(s0, s1x, s1y, s2v, K2h[o], K1h[o], D2h[o], odd_transposed(D2h, kx, ky, L, H), s2);
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    PR[(q * nc + c) * L + ky] = conv_product(q, s0, s1x, s1y, K2h, Keh, D2h, Deh, kx, ky, L, H);
            }
            __syncthreads();
            float2* R2 = fft_lines(PR, PP, 6 * nc, L, G, stw);
            for (int idx = threadIdx.x; idx < 6 * nc * M; idx += blockDim.x) {
                const int y = idx / (6 * nc), r = idx - y * (6 * nc);
                const int q = r / nc, c = r - q * nc;
                ucol[(int64_t)q * MH + (int64_t)y * H + k0 + c] = conj2(R2[r * L + y]);
            }
        }
    } else {
        // Long lines: four kept spectra + two work lines per column.
        const int cap = line_cap(sm_f2, L, 6);
        float2* buf[6];
        for (int i = 0; i < 6; ++i) buf[i] = smf + L + (size_t)i * cap * L;
        for (int k0 = beg; k0 < end; k0 += cap) {
            const int nl = min(cap, end - k0);
            float2* spec[4];
            float2* pool[6] = {buf[0], buf[1], buf[2], buf[3], buf[4], buf[5]};
            for (int gsel = 0; gsel < 4; ++gsel) {
                float2* a = pool[gsel];
                float2* b = pool[gsel + 1];
                __syncthreads();
                for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
                    const int y = idx / nl, line = idx - y * nl;
                    a[line * L + y] =
                        y < M ? srow[(int64_t)gsel * MH + (int64_t)y * H + k0 + line] : make_float2(0.f, 0.f);
                }
                __syncthreads();
                float2* r = fft_lines(a, b, nl, L, G, stw);
                spec[gsel] = r;
                pool[gsel] = r;
                pool[gsel + 1] = (r == a) ? b : a;
            }
            float2* wa = pool[4];
            float2* wb = pool[5];
            for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
                const int ky = idx / nl, line = idx - ky * nl;
                const int kx = k0 + line;
                const int64_t o = (int64_t)ky * H + kx;
                const double wgt = (kx == 0 || 2 * kx == L) ? 1.0 : 2.0;
                zacc += wgt * z_term(spec[0][line * L + ky], spec[1][line * L + ky], spec[2][line * L + ky],
                                     spec[3][line * L + ky], K2h[o], K1h[o], D2h[o],
                                     odd_transposed(D2h, kx, ky, L, H), s2);
            }
            for (int q = 0; q < 6; ++q) {
                __syncthreads();
                for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
                    const int ky = idx / nl, line = idx - ky * nl;
                    wa[line * L + ky] = conv_product(q, spec[0][line * L + ky], spec[1][line * L + ky],
                                                     spec[2][line * L + ky], K2h, Keh, D2h, Deh, k0 + line, ky, L, H);
                }
                __syncthreads();
                float2* r = fft_lines(wa, wb, nl, L, G, stw);
                for (int idx = threadIdx.x; idx < nl * M; idx += blockDim.x) {
                    const int y = idx / nl, line = idx - y * nl;
                    ucol[(int64_t)q * MH + (int64_t)y * H + k0 + line] = conj2(r[line * L + y]);
                }
            }
        }
    }
    red[threadIdx.x] = zacc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        zblk[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(&Gp->ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double v = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += ((volatile double*)zblk)[b];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double Z = red[0] - (double)n;
            Gp->Z = Z;
            Gp->SoZ = (float)(Gp->S / Z);
        }
    }
}

// Inverse row FFTs, three packed lines per row (U0 + i U1, U2 + i U3,
// U4 + i U5), each half spectrum extended by Hermitian symmetry.  Fields per
// node: f0 = F0, f1 = Vx, f2 = Vy, f3 = Fe0, f4 = Vex, f5 = Vey, f6 = f7 = 0.
// Also clears the charge grid (its readers have finished) for the next spread.
__global__ void k_conv_rows_inv(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                                const float2* __restrict__ ucol, float* __restrict__ fields,
                                long long* __restrict__ wfix, float4* __restrict__ wflt, int plain, int sm_f2)
{
    extern __shared__ float2 smf[];
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    const int cap = line_cap(sm_f2, L, 2);
    float2* stw = smf;
    float2* A = smf + L;
    float2* B = A + (size_t)cap * L;
    load_tw(stw, tw, L);
    const int64_t MH = (int64_t)M * H;
    int beg, end;
    block_range(3 * M, beg, end);  // unit = (pair, row)
    for (int u0 = beg; u0 < end; u0 += cap) {
        const int nl = min(cap, end - u0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
            const int line = idx / L, k = idx - line * L;
            const int u = u0 + line, pr = u / M, row = u - pr * M;
            const float2* ua = ucol + (int64_t)(2 * pr) * MH + (int64_t)row * H;
            const float2* ub = ua + MH;
            float2 a, b;
            if (k < H) {
                a = ua[k];
                b = ub[k];
            } else {
                a = conj2(ua[L - k]);
                b = conj2(ub[L - k]);
            }
            A[line * L + k] = conj2(make_float2(a.x - b.y, a.y + b.x));  // conj(a + i b)
        }
        __syncthreads();
        float2* R = fft_lines(A, B, nl, L, G, stw);
        for (int idx = threadIdx.x; idx < nl * M; idx += blockDim.x) {
            const int line = idx / M, x = idx - line * M;
            const int u = u0 + line, pr = u / M, row = u - pr * M;
            const float2 v = conj2(R[line * L + x]);
            float* f = fields + ((int64_t)row * M + x) * kFieldStride;
            if (pr == 0) { f[0] = v.x; f[3] = v.y; f[6] = 0.f; f[7] = 0.f; }
            else if (pr == 1) { f[1] = v.x; f[2] = v.y; }
            else { f[4] = v.x; f[5] = v.y; }
        }
    }
    for (int u = beg; u < end; ++u) {
        if (u >= M) break;  // units (0, row) cover every row once
        for (int x = threadIdx.x; x < M; x += blockDim.x) {
            const int64_t node = (int64_t)u * M + x;
            if (plain) wflt[node] = make_float4(0.f, 0.f, 0.f, 0.f);
            else {
                long long* q = wfix + node * 4;
                q[0] = 0; q[1] = 0; q[2] = 0; q[3] = 0;
            }
        }
    }
}

__global__ void k_bounds_init(int32_t* b)
{
    b[0] = f2ord(INFINITY);
    b[1] = f2ord(-INFINITY);
}

__global__ void k_bounds(const float2* __restrict__ Y, int32_t n, int32_t* __restrict__ b)
{
    __shared__ float smin[32], smax[32];
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = Y[i];
        mn = fminf(mn, fminf(p.x, p.y));
        mx = fmaxf(mx, fmaxf(p.x, p.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        smin[w] = mn;
        smax[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            mn = fminf(mn, smin[i]);
            mx = fmaxf(mx, smax[i]);
        }
        atomicMin(&b[0], f2ord(mn));
        atomicMax(&b[1], f2ord(mx));
    }
}

__global__ void k_psum(const float* __restrict__ v, const int64_t* __restrict__ nnz_ptr, double* __restrict__ sblk,
                       GridDev* G)
{
    __shared__ double red[256];
    __shared__ bool last;
    const int64_t nnz = *nnz_ptr;
    double a = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        a += (double)v[e];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sblk[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(&G->ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) t += ((volatile double*)sblk)[b];
        G->S = t;
        G->ticket = 0;
    }
}

constexpr int kFftThreads = 256;
constexpr int kPsumBlocks = 304;

// Shared memory of the spread: the fixed-point tile, the item's points and
// their boxes, box offsets and cursors.
size_t spread_smem_bytes()
{
    return (size_t)kMaxTileNodes * kMaxTileNodes * 4 * sizeof(long long) +
           (size_t)kSpreadChunk * (sizeof(float2) + sizeof(int)) + (size_t)(2 * kMaxTileBoxes + 1) * sizeof(int);
}

// Room for the twiddles plus six lines of the longest length (the column
// pass keeps four spectra and two work lines), at least 64 KB.
size_t fft_smem_bytes(int Lmax) { return std::max<size_t>(64 * 1024, (size_t)7 * Lmax * 8); }

}  // namespace

IterShape iter_shape(int32_t n, const ltsnet_params* p)
{
    IterShape sh;
    sh.n = n;
    sh.P = p->nodes_per_box;
    sh.max_boxes = p->max_boxes;
    sh.Mmax = p->max_boxes * p->nodes_per_box;
    sh.Lmax = 2 * sh.Mmax;
    sh.tiles_max = kMaxTiles;
    sh.items_max = (int64_t)kMaxTiles * kMaxTiles + (int64_t)n / kSpreadChunk + 2;
    return sh;
}

IterWs iter_carve(Carve& c, const IterShape& sh)
{
    IterWs w;
    const int64_t T = (int64_t)sh.tiles_max * sh.tiles_max;
    const int64_t MM = (int64_t)sh.Mmax * sh.Mmax;
    w.st = c.take<StatusBlock>(1);
    w.g = c.take<GridDev>(1);
    w.bounds = c.take<int32_t>(4);
    w.tw = c.take<float2>(kLMax);
    w.tile_cnt = c.take<int32_t>(T);
    w.tile_off = c.take<int32_t>(T + 1);
    w.tile_cur = c.take<int32_t>(T);
    w.items = c.take<int4>(sh.items_max);
    w.binned = c.take<float2>(sh.n);
    w.wfix = c.take<long long>(4 * MM);
    w.wflt = c.take<float4>(MM);
    const int64_t LH = (int64_t)sh.Lmax * (sh.Lmax / 2 + 1);
    const int64_t MH = (int64_t)sh.Mmax * (sh.Lmax / 2 + 1);
    w.krow = c.take<float2>(3 * LH);
    w.khat = c.take<float>(5 * LH);
    w.srow = c.take<float2>(4 * MH);
    w.ucol = c.take<float2>(6 * MH);
    w.fields = c.take<float>(MM * kFieldStride);
    w.zblk = c.take<double>(1024);
    w.sblk = c.take<double>(1024);
    w.yalt = c.take<float2>(sh.n);
    w.phi = c.take<float>((int64_t)sh.n * 8);
    w.attr = c.take<float2>(sh.n);
    return w;
}

cudaError_t launch_bounds_init(const IterWs& w, const float2* Y, int32_t n, int parity, cudaStream_t s)
{
    int32_t* b = w.bounds + 2 * parity;
    k_bounds_init<<<1, 1, 0, s>>>(b);
    int64_t blocks = ((int64_t)n + 255) / 256;
    if (blocks > kSMs * 4) blocks = kSMs * 4;
    if (blocks < 1) blocks = 1;
    k_bounds<<<(unsigned)blocks, 256, 0, s>>>(Y, n, b);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_psum(const IterWs& w, const int64_t* P_row, int32_t n, const float* P_val, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(&w.g->ticket, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_psum<<<kPsumBlocks, 256, 0, s>>>(P_val, P_row + n, w.sblk, w.g);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_grid_phase(const IterWs& w, const IterShape& sh, const ltsnet_params* p, const float2* Y,
                              int parity, bool plain, cudaStream_t s)
{
    const int32_t n = sh.n;
    const int P = sh.P;
    k_setup<<<16, 256, 0, s>>>(w.bounds + 2 * parity, w.bounds + 2 * (parity ^ 1), w.g, w.tw, w.tile_cnt, n,
                               p->box_width_max, p->min_boxes, p->max_boxes, P);
    count_launches(1);
    profile_start(LTSNET_KERNEL_SPREAD, s);
    const int64_t T = (int64_t)sh.tiles_max * sh.tiles_max;
    if (plain) {
        int64_t blocks = ((int64_t)n + 255) / 256;
        if (blocks > kSMs * 8) blocks = kSMs * 8;
        if (blocks < 1) blocks = 1;
        switch (P) {
            case 2: k_spread_atomic<2><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
            case 3: k_spread_atomic<3><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
            case 4: k_spread_atomic<4><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
            default: k_spread_atomic<5><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
        }
        count_launches(1);
    } else {
        int64_t blocks = ((int64_t)n + 255) / 256;
        if (blocks > kSMs * 4) blocks = kSMs * 4;
        if (blocks < 1) blocks = 1;
        const size_t sm1 = (size_t)T * 4;
        k_bin_count<<<(unsigned)blocks, 256, sm1, s>>>(Y, n, w.g, w.tile_cnt);
        k_bin_plan<<<1, 1024, 0, s>>>(w.g, w.tile_cnt, w.tile_off, w.tile_cur, w.items, kSpreadChunk);
        int64_t sblocks = ((int64_t)n + 256 * 8 - 1) / (256 * 8);
        if (sblocks < 1) sblocks = 1;
        k_bin_scatter<<<(unsigned)sblocks, 256, 2 * sm1, s>>>(Y, n, w.g, w.tile_cur, w.binned);
        const size_t sm2 = spread_smem_bytes();
        switch (P) {
            case 2: k_spread_tiles<2><<<kSMs * 4, 256, sm2, s>>>(w.binned, w.g, w.items, w.wfix); break;
            case 3: k_spread_tiles<3><<<kSMs * 4, 256, sm2, s>>>(w.binned, w.g, w.items, w.wfix); break;
            case 4: k_spread_tiles<4><<<kSMs * 4, 256, sm2, s>>>(w.binned, w.g, w.items, w.wfix); break;
            default: k_spread_tiles<5><<<kSMs * 4, 256, sm2, s>>>(w.binned, w.g, w.items, w.wfix); break;
        }
        count_launches(4);
    }
    profile_stop(LTSNET_KERNEL_SPREAD, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    profile_start(LTSNET_KERNEL_CONV, s);
    const size_t fsm = fft_smem_bytes(sh.Lmax);
    const int f2 = (int)(fsm / sizeof(float2));
    k_spec_rows<<<kSMs, kFftThreads, fsm, s>>>(w.g, w.tw, p->eps, w.krow, f2);
    k_spec_cols<<<kSMs, kFftThreads, fsm, s>>>(w.g, w.tw, w.krow, w.khat, f2);
    k_conv_rows_fwd<<<kSMs, kFftThreads, fsm, s>>>(w.g, w.tw, w.wfix, w.wflt, plain ? 1 : 0, w.srow, f2);
    k_conv_cols<<<kSMs, kFftThreads, fsm, s>>>(w.g, w.tw, w.srow, w.khat, w.ucol, w.zblk, n, f2);
    k_conv_rows_inv<<<kSMs, kFftThreads, fsm, s>>>(w.g, w.tw, w.ucol, w.fields, w.wfix, w.wflt, plain ? 1 : 0, f2);
    count_launches(5);
    profile_stop(LTSNET_KERNEL_CONV, s);
    return cudaGetLastError();
}

cudaError_t grid_set_smem_attrs()
{
    const int fsm = (int)fft_smem_bytes(kLMax);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_spec_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_spec_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    const int sm2 = (int)spread_smem_bytes();
    if ((e = cudaFuncSetAttribute(k_spread_tiles<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2))) return e;
    if ((e = cudaFuncSetAttribute(k_spread_tiles<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2))) return e;
    if ((e = cudaFuncSetAttribute(k_spread_tiles<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2))) return e;
    if ((e = cudaFuncSetAttribute(k_spread_tiles<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2))) return e;
    // binning: one int (count) or two (count, base) per tile
    const int bins = kMaxTiles * kMaxTiles * 4;
    if ((e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, bins))) return e;
    if ((e = cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * bins))) return e;
    return cudaSuccess;
}

}  // namespace lt
