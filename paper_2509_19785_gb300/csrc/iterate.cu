// The per-iteration gradient and the descent loop (Alg. 3 loop body).
//
// k_fused (optimised form): one warp per 32 consecutive vertices.
//   Attraction (Eq. 6, first term): the warp walks the 32 rows of P four at a
//   time, 8 lanes per row, each lane reading 4 entries (value, column) per
//   vector load from the packed layout built by k_pack_rows (or from CSR
//   with int32 columns); the lanes' partial sums go to shared memory and
//   each row's lane adds its row's 8 partials.
//   Then every lane, for its own vertex: gathers the interpolated repulsion
//   sum R_i (Sec. 2.3) and entropy sum E_i (Eq. 8, repulsive reading) from
//   the P x P nodes of its box, adds the compression (lambda_c/n) X_i
//   (Eq. 1), assembles the gradient and applies the momentum/gain step,
//   writing the new layout to the other ping-pong buffer and folding it into
//   the bounds of the next grid.
// Plain form: the same arithmetic split into a gather kernel, an attraction
// kernel and an update kernel with intermediates in global memory.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "iter.cuh"
#include "prims.cuh"

namespace lt {
namespace {

struct Coeffs {
    float a_att, a_rep, a_cmp, a_ent;
};

__device__ __forceinline__ Coeffs coeffs(const GridDev* G, const Stage& st)
{
    Coeffs k;
    k.a_att = st.a_att;
    k.a_rep = st.a_rep * G->SoZ;
    k.a_cmp = st.a_cmp;
    k.a_ent = st.a_ent;
    return k;
}

// Sum over CSR row [s0, e0) of p_ij (X_i - X_j) / (1 + |X_i - X_j|^2) by one
// warp: lane l handles entries eb + 4l .. eb + 4l + 3 for eb from s0 rounded
// down to a multiple of 4, so the int4/float4 loads are aligned.
__device__ __forceinline__ float2 warp_row_attraction(const int32_t* __restrict__ P_col,
                                                      const float* __restrict__ P_val, int64_t nnz, int64_t s0,
                                                      int64_t e0, float xi, float yi, const float2* __restrict__ Y,
                                                      int32_t n, int lane, StatusBlock* status)
{
    float ax = 0.f, ay = 0.f;
    for (int64_t eb = s0 & ~(int64_t)3; eb < e0; eb += 128) {
        const int64_t e = eb + 4 * lane;
        if (e < e0) {
            int cj[4];
            float pv[4];
            if (e + 3 < nnz) {
                const int4 c4 = __ldg((const int4*)(P_col + e));
                const float4 v4 = __ldg((const float4*)(P_val + e));
                cj[0] = c4.x; cj[1] = c4.y; cj[2] = c4.z; cj[3] = c4.w;
                pv[0] = v4.x; pv[1] = v4.y; pv[2] = v4.z; pv[3] = v4.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    cj[q] = (e + q < nnz) ? P_col[e + q] : 0;
                    pv[q] = (e + q < nnz) ? P_val[e + q] : 0.f;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t idx = e + q;
                if (idx >= s0 && idx < e0) {
                    if ((unsigned)cj[q] >= (unsigned)n) {
                        record_error(status, LTSNET_ERR_BAD_GRAPH, cj[q]);
                        continue;
                    }
                    const float2 yj = __ldg(Y + cj[q]);
                    const float dx = xi - yj.x, dy = yi - yj.y;
                    const float w = pv[q] / (1.0f + dx * dx + dy * dy);
                    ax += w * dx;
                    ay += w * dy;
                }
            }
        }
    }
    return make_float2(warp_sum(ax), warp_sum(ay));
}

// Interpolated repulsion and entropy sums of one point (node-local form):
//   R = s sum_ab L_a L_b [e . F0 + V],  E = s sum_ab L_a L_b [e . Fe0 + Ve]
// with e the point's offset from node (a, b) in node spacings.
struct Sums {
    float2 R, E;
};

template <int P>
__device__ __forceinline__ Sums gather_sums(float2 p, const GridDev* G, const float* __restrict__ fields)
{
    const int M = G->M;
    int bx, by;
    float ux, uy;
    local_coords(p, G, bx, by, ux, uy);
    float wx[P], wy[P];
    lagrange<P>(ux, wx);
    lagrange<P>(uy, wy);
    float rx = 0.f, ry = 0.f, ex = 0.f, ey = 0.f;
#pragma unroll
    for (int b = 0; b < P; ++b)
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const float w = wx[a] * wy[b];
            const float dx = ux - ((float)a + 0.5f), dy = uy - ((float)b + 0.5f);
            const float4* nd = (const float4*)(fields + ((int64_t)(P * by + b) * M + (P * bx + a)) * kFieldStride);
            const float4 u = __ldg(nd), v = __ldg(nd + 1);  // (F0, Vx, Vy, Fe0), (Vex, Vey, -, -)
            rx += w * (dx * u.x + u.y);
            ry += w * (dy * u.x + u.z);
            ex += w * (dx * u.w + v.x);
            ey += w * (dy * u.w + v.y);
        }
    const float s = G->s;
    Sums r;
    r.R = make_float2(s * rx, s * ry);
    r.E = make_float2(s * ex, s * ey);
    return r;
}

__device__ __forceinline__ float sgn(float v) { return (float)((v > 0.f) - (v < 0.f)); }

// Gradient of vertex i and (optionally) its momentum/gain step.
struct PointOut {
    float2 g, A, R, E;
};

__device__ __forceinline__ PointOut point_gradient(float2 p, float2 A, const Sums& F, const Coeffs& k)
{
    PointOut o;
    o.A = A;
    o.R = F.R;
    o.E = F.E;
    o.g.x = k.a_att * A.x - k.a_rep * o.R.x + k.a_cmp * p.x - k.a_ent * o.E.x;
    o.g.y = k.a_att * A.y - k.a_rep * o.R.y + k.a_cmp * p.y - k.a_ent * o.E.y;
    return o;
}

__device__ __forceinline__ float2 step(float2 p, float2 g, float2& u, float2& gn, const Stage& st)
{
    gn.x = (sgn(g.x) != sgn(u.x)) ? gn.x + 0.2f : gn.x * 0.8f;
    gn.y = (sgn(g.y) != sgn(u.y)) ? gn.y + 0.2f : gn.y * 0.8f;
    gn.x = fmaxf(gn.x, 0.01f);
    gn.y = fmaxf(gn.y, 0.01f);
    u.x = st.momentum * u.x - st.lr * gn.x * g.x;
    u.y = st.momentum * u.y - st.lr * gn.y * g.y;
    return make_float2(p.x + u.x, p.y + u.y);
}

__device__ __forceinline__ void block_bounds(float mn, float mx, int32_t* bounds_next)
{
    __shared__ float smn[32], smx[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        smn[w] = mn;
        smx[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            mn = fminf(mn, smn[i]);
            mx = fmaxf(mx, smx[i]);
        }
        if (mn <= mx) {
            atomicMin(&bounds_next[0], f2ord(mn));
            atomicMax(&bounds_next[1], f2ord(mx));
        }
    }
}

constexpr int kFusedThreads = 256;
constexpr int kRowLanes = 8;     // lanes per CSR row in the attraction pass
constexpr int kWin = 128;        // CSR entries of a row taken per round (longer rows: the rest directly)
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kHeavyRow = 2048;  // longer rows of P are summed in chunks by k_attr_chunks
constexpr int kChunk = 2048;     // entries per chunk
constexpr int kTailBatch = 8;    // entries per lane in flight past a row's window

// Rows of P longer than kHeavyRow (hubs of scale-free graphs can sit in a
// large part of all neighbour lists): their attraction sums are computed in
// chunks of kChunk entries by whole warps, and the fused kernel adds a row's
// chunk sums in chunk order (deterministic).  hbase[row] is the row's first
// chunk; read only for rows longer than kHeavyRow.
struct HeavyRows {
    const int32_t* hbase = nullptr;
    const int32_t* crow = nullptr;
    const int64_t* cstart = nullptr;
    float2* partial = nullptr;
    int32_t nchunks = 0;
};

// P as the point phase streams it: row pointers, int32 columns (CSR or the
// int32 packed layout) or int16 offsets (the int16 packed layout), values,
// the format (kFmt* below) and the long rows' chunk lists.
struct PStream {
    const int64_t* row = nullptr;
    const int32_t* col = nullptr;
    const int16_t* d16 = nullptr;
    const float* val = nullptr;
    int fmt = 0;
    HeavyRows hr;
};

// A caller's P: CSR with int32 columns, no chunk lists.
PStream csr_stream(const int64_t* P_row, const int32_t* P_col, const float* P_val)
{
    PStream sp;
    sp.row = P_row;
    sp.col = P_col;
    sp.val = P_val;
    return sp;
}

// Paired FP32 arithmetic (sm_100 family): each half is the IEEE
// round-to-nearest result of the scalar operation, so these give the same
// bits as two scalar instructions in one issue.
__device__ __forceinline__ unsigned long long pack2(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
// a - b, componentwise
__device__ __forceinline__ float2 sub_x2(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
// (w, w) * d + c, componentwise
__device__ __forceinline__ float2 fma_x2(float w, float2 d, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pack2(make_float2(w, w))), "l"(pack2(d)), "l"(pack2(c)));
    return unpack2(r);
}

// 1/x to within about one unit in the last place (the SFU reciprocal);
// x >= 1 here.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}


// Per lane and round: 16 consecutive slots of its row's window (4 chunks of
// 4 entries), columns as int32 indices or, for the library's own P, as int16
// offsets from the row (col - row).
// The raw words are kept until the round that uses them: decoding them at
// load time would stall the warp on the load right away.
struct Window {
    int4 c[4];      // int32 columns, or int16 offsets in (x, y) of each chunk
    float4 v[4];    // P values
};

// Formats P is streamed in by the point phase: CSR with int32 columns (a
// caller's P), or the packed layout of k_pack_rows with int16 column offsets
// from the row or with int32 columns.
constexpr int kFmtCsr = 0;
constexpr int kFmtPk16 = 1;
constexpr int kFmtPk32 = 2;

// int32 columns of chunk u of a window (CSR form)
__device__ __forceinline__ void window_cols(const Window& w, int u, int* cc)
{
    cc[0] = w.c[u].x;
    cc[1] = w.c[u].y;
    cc[2] = w.c[u].z;
    cc[3] = w.c[u].w;
}

// Window end: the row's end, or its start for a long row (summed in chunks
// beforehand), so that the window holds no entry of it.
__device__ __forceinline__ int64_t window_end(const int32_t* hbase, int64_t s0, int64_t e0)
{
    return hbase != nullptr && e0 - s0 > kHeavyRow ? s0 : e0;
}

// Window start: the row start, which the packed layouts keep a multiple of 4
// entries; for CSR the row start rounded down to a multiple of 4 so that
// every vector load is aligned.
template <int FMT>
__device__ __forceinline__ int64_t window_start(int64_t s0)
{
    return FMT != kFmtCsr ? s0 : (s0 & ~(int64_t)3);
}

// Load the lane's slots j = 32 u + 4 gl + q (u, q < 4) of the window starting
// at eb: vector loads that bypass L1 (the stream is read once), scalar
// loads where a vector would pass the end of the arrays (nnz), nothing past
// the row's end e0.
template <int FMT>
__device__ __forceinline__ void load_window(Window& w, const int32_t* __restrict__ P_col,
                                            const int16_t* __restrict__ P_d16, const float* __restrict__ P_val,
                                            int64_t nnz, int64_t eb, int64_t e0, int rowi, int gl)
{
    constexpr bool D16 = FMT == kFmtPk16;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t e = eb + 32 * u + 4 * gl;
        if (e < e0 && e + 4 <= nnz) {
            w.v[u] = __ldcs((const float4*)(P_val + e));
            if (D16) {
                const uint2 d = __ldcs((const uint2*)(P_d16 + e));
                w.c[u] = make_int4((int)d.x, (int)d.y, 0, 0);
            } else {
                w.c[u] = __ldcs((const int4*)(P_col + e));
            }
        } else {
            // near the end of the arrays or past the row: scalar loads (rare),
            // missing entries as column offset 0 / the row itself, weight 0
            float vv[4];
            int cv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool ok = e + q < e0 && e + q < nnz;
                vv[q] = ok ? P_val[e + q] : 0.f;
                cv[q] = ok ? (D16 ? (int)(uint16_t)P_d16[e + q] : P_col[e + q]) : (D16 ? 0 : rowi);
            }
            w.v[u] = make_float4(vv[0], vv[1], vv[2], vv[3]);
            w.c[u] = D16 ? make_int4((int)((unsigned)cv[0] | ((unsigned)cv[1] << 16)),
                                     (int)((unsigned)cv[2] | ((unsigned)cv[3] << 16)), 0, 0)
                         : make_int4(cv[0], cv[1], cv[2], cv[3]);
        }
    }
}

// One warp per 32 consecutive vertices.  Attraction (Eq. 6, first term) in 8
// rounds of 4 rows, one row per 8-lane group, each lane taking 16 slots of
// its row's 128-entry window; the next round's window is loaded into
// registers before this round gathers its neighbours' coordinates, so the
// HBM stream overlaps the gathers.  Entries past the window (rows longer
// than it) are read directly.  Row r's sum goes to lane r, which then
// finishes its vertex: interpolated repulsion and entropy (gather from the
// grid), compression, gradient, momentum/gain step, bounds of the next grid.
template <int P, bool UPDATE, int FMT>
__device__ __forceinline__ void
    k_fused_body(const int64_t* __restrict__ P_row, const int32_t* __restrict__ P_col, const int16_t* __restrict__ P_d16,
            const float* __restrict__ P_val,
            int32_t n, const float2* __restrict__ Y, float2* __restrict__ Ynew, float2* __restrict__ upd,
            float2* __restrict__ gains, const GridDev* __restrict__ G, const float* __restrict__ fields, Stage st,
            int32_t* __restrict__ bounds_next, float2* __restrict__ grad_out, float* __restrict__ parts,
            StatusBlock* status, const int32_t* __restrict__ hbase, const float2* __restrict__ hpartial)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane >> 3, gl = lane & 7;
    __shared__ float2 part_all[kFusedWarps][256];
    float2* part = part_all[wib];
    const Coeffs k = coeffs(G, st);
    const int64_t nnz = P_row[n];
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t g0 = ((int64_t)blockIdx.x * kFusedWarps + wib) * 32; g0 < n;
         g0 += (int64_t)gridDim.x * kFusedWarps * 32) {
        const int64_t row = g0 + lane;
        const bool has = row < n;
        const float2 yi = has ? Y[row] : make_float2(0.f, 0.f);
        const int64_t rs = has ? P_row[row] : 0;
        const int64_t re = has ? P_row[row + 1] : 0;
        // row bounds as 32-bit offsets from the group's first row (the
        // arrays have fewer than 2^32 entries): one shuffle each
        const int64_t base = __shfl_sync(FULL, rs, 0);
        const uint32_t rs32 = has ? (uint32_t)(rs - base) : 0u, re32 = has ? (uint32_t)(re - base) : 0u;
        float2 A = make_float2(0.f, 0.f);
        Window nxt;
        // bounds of the next round's row, shuffled once and kept for its round
        int64_t ns0 = base + __shfl_sync(FULL, rs32, grp), ne0 = base + __shfl_sync(FULL, re32, grp);
        load_window<FMT>(nxt, P_col, P_d16, P_val, nnz, window_start<FMT>(ns0), window_end(hbase, ns0, ne0),
                         (int)(g0 + grp), gl);
#pragma unroll 1
        for (int rr = 0; rr < 8; ++rr) {
            const Window cur = nxt;
            const int src = rr * 4 + grp;
            const int rowi = (int)(g0 + src);
            const int64_t s0 = ns0, e0r = ne0;
            if (rr < 7) {
                const int nsrc = src + 4;
                ns0 = base + __shfl_sync(FULL, rs32, nsrc);
                ne0 = base + __shfl_sync(FULL, re32, nsrc);
                load_window<FMT>(nxt, P_col, P_d16, P_val, nnz, window_start<FMT>(ns0), window_end(hbase, ns0, ne0),
                                 rowi + 4, gl);
            }
            const float xi = __shfl_sync(FULL, yi.x, src), yv = __shfl_sync(FULL, yi.y, src);
            const bool heavy = hbase != nullptr && e0r - s0 > kHeavyRow;  // summed in chunks already
            const int64_t e0 = heavy ? s0 : e0r;
            const int64_t eb = window_start<FMT>(s0);
            const int off = (int)(s0 - eb);  // leading slots that belong to the previous row
            const int64_t len = e0 - eb;     // slots from len on belong to the next rows
            float2 acc = make_float2(0.f, 0.f);
            float2 yj[4][4];
            float pv[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 32 * u + 4 * gl;
                const float vv[4] = {cur.v[u].x, cur.v[u].y, cur.v[u].z, cur.v[u].w};
                if (FMT == kFmtPk16) {
                    // Packed rows: every slot gathers.  Slots past the row's
                    // window (past its end, or a long row's) were loaded as
                    // offset 0 and weight 0, like the pads of a packed row,
                    // so they read the point itself and add nothing; and
                    // k_pack_rows checked every column against [0, n).
                    const float2* yr = Y + rowi;
                    const int o[4] = {(int)(int16_t)(cur.c[u].x & 0xffff), cur.c[u].x >> 16,
                                      (int)(int16_t)(cur.c[u].y & 0xffff), cur.c[u].y >> 16};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        yj[u][q] = __ldg(yr + o[q]);
                        pv[u][q] = vv[q];
                    }
                    continue;
                }
                if (FMT == kFmtPk32) {
                    // packed rows with int32 columns: as above, slots past
                    // the window hold the row itself with weight 0
                    const int cq[4] = {cur.c[u].x, cur.c[u].y, cur.c[u].z, cur.c[u].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        yj[u][q] = __ldg(Y + cq[q]);
                        pv[u][q] = vv[q];
                    }
                    continue;
                }
                int cc[4];
                window_cols(cur, u, cc);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // Slots of other rows get weight 0 and no gather (the
                    // point itself stands in); the clamp keeps the gathers
                    // of an invalid P in range (k_check_cols reports it).
                    const bool own = j + q >= off && j + q < len;
                    const unsigned c = min((unsigned)cc[q], (unsigned)(n - 1));
                    yj[u][q] = own ? __ldg(Y + c) : make_float2(xi, yv);
                    pv[u][q] = own ? vv[q] : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 d = sub_x2(make_float2(xi, yv), yj[u][q]);
                    const float w = pv[u][q] * rcp_approx(__fmaf_rn(d.y, d.y, __fmaf_rn(d.x, d.x, 1.0f)));
                    acc = fma_x2(w, d, acc);
                }
            // entries past the window: kTailBatch per lane at a time, all
            // loads, then all gathers, issued before any is used
            for (int64_t eb2 = eb + kWin + gl; eb2 < e0; eb2 += kRowLanes * kTailBatch) {
                int tc[kTailBatch];
                float tv[kTailBatch];
#pragma unroll
                for (int t = 0; t < kTailBatch; ++t) {
                    const int64_t e = eb2 + kRowLanes * t;
                    const bool ok = e < e0;
                    tc[t] = ok ? (FMT == kFmtPk16 ? rowi + (int)__ldg(P_d16 + e) : __ldg(P_col + e)) : rowi;
                    tv[t] = ok ? __ldg(P_val + e) : 0.f;
                }
                float2 tq[kTailBatch];
#pragma unroll
                for (int t = 0; t < kTailBatch; ++t) tq[t] = __ldg(Y + min((unsigned)tc[t], (unsigned)(n - 1)));
#pragma unroll
                for (int t = 0; t < kTailBatch; ++t) {
                    const float2 d = sub_x2(make_float2(xi, yv), tq[t]);
                    const float w = tv[t] * rcp_approx(__fmaf_rn(d.y, d.y, __fmaf_rn(d.x, d.x, 1.0f)));
                    acc = fma_x2(w, d, acc);
                }
            }
            if (heavy) {
                const int b = hbase[rowi];
                const int nc = (int)((e0r - s0 + kChunk - 1) / kChunk);
                for (int c = gl; c < nc; c += kRowLanes) {
                    const float2 q = hpartial[b + c];
                    acc.x += q.x;
                    acc.y += q.y;
                }
            }
            // lane (group g, gl) of round rr holds a partial sum of row
            // rr * 4 + g: kept at slot row * 8 + gl = rr * 32 + lane
            part[rr * 32 + lane] = acc;
        }
        __syncwarp();
        {
            // row `lane` adds its 8 partials, starting at slot lane / 2 of
            // its row: the 32 lanes of one step then hit 16 distinct pairs of
            // banks (two lanes each, two wavefronts)
            float2 t = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kRowLanes; ++k) {
                const float2 q = part[lane * 8 + ((k + (lane >> 1)) & 7)];
                t.x += q.x;
                t.y += q.y;
            }
            A = t;
        }
        __syncwarp();
        if (has) {
            const Sums F = gather_sums<P>(yi, G, fields);
            const PointOut o = point_gradient(yi, A, F, k);
            if (UPDATE) {
                float2 u = upd[row], gn = gains[row];
                const float2 yn = step(yi, o.g, u, gn, st);
                upd[row] = u;
                gains[row] = gn;
                Ynew[row] = yn;
                if (!(isfinite(yn.x) && isfinite(yn.y))) record_error(status, LTSNET_ERR_NONFINITE, (int32_t)row);
                mn = fminf(mn, fminf(yn.x, yn.y));
                mx = fmaxf(mx, fmaxf(yn.x, yn.y));
            } else {
                grad_out[row] = o.g;
                if (!(isfinite(o.g.x) && isfinite(o.g.y))) record_error(status, LTSNET_ERR_NONFINITE, (int32_t)row);
                if (parts) {
                    float* q = parts + row * 6;
                    q[0] = o.A.x; q[1] = o.A.y; q[2] = o.R.x; q[3] = o.R.y; q[4] = o.E.x; q[5] = o.E.y;
                }
            }
        }
    }
    if (UPDATE) block_bounds(mn, mx, bounds_next);
}

template <int P, bool UPDATE, int FMT>
__global__ void __launch_bounds__(kFusedThreads, 2)
    k_fused(const int64_t* __restrict__ P_row, const int32_t* __restrict__ P_col, const int16_t* __restrict__ P_d16,
            const float* __restrict__ P_val,
            int32_t n, const float2* __restrict__ Y, float2* __restrict__ Ynew, float2* __restrict__ upd,
            float2* __restrict__ gains, const GridDev* __restrict__ G, const float* __restrict__ fields, Stage st,
            int32_t* __restrict__ bounds_next, float2* __restrict__ grad_out, float* __restrict__ parts,
            StatusBlock* status, const int32_t* __restrict__ hbase, const float2* __restrict__ hpartial)
{
    k_fused_body<P, UPDATE, FMT>(P_row, P_col, P_d16, P_val, n, Y, Ynew, upd, gains, G, fields, st, bounds_next,
                                 grad_out, parts, status, hbase, hpartial);
}

// The fused point phase of one iteration for every graph of a batch (graph =
// blockIdx.y), layouts by parity as in one_iteration.
template <int P, int FMT>
__global__ void __launch_bounds__(kFusedThreads, 2) k_fused_b(const BatchGraph* __restrict__ bg, int parity)
{
    const BatchGraph& b = bg[blockIdx.y];
    const float2* cur = parity ? b.w.yalt : b.Y;
    float2* nxt = parity ? b.Y : b.w.yalt;
    k_fused_body<P, true, FMT>(b.P_row, b.P_col, b.P_d16, b.P_val, b.n, cur, nxt, b.upd, b.gains, b.w.g, b.w.fields,
                               b.st, b.w.bounds + 2 * (parity ^ 1), nullptr, nullptr, b.w.st, b.hbase, b.hpartial);
}

constexpr size_t kFusedSmem = 0;  // the windows live in registers

// Attraction sums of the chunks of the long rows: one warp per chunk of
// kChunk entries of one row, lanes striding over the entries.
constexpr int kChunkBatch = 8;
template <bool D16>
__device__ __forceinline__ void k_attr_chunks_body(const int64_t* __restrict__ P_row,
                                                   const int32_t* __restrict__ P_col,
                                                   const int16_t* __restrict__ P_d16,
                                                   const float* __restrict__ P_val, int32_t n,
                                                   const float2* __restrict__ Y, const int32_t* __restrict__ crow,
                                                   const int64_t* __restrict__ cstart, int32_t nchunks,
                                                   float2* __restrict__ partial)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += nw) {
        const int32_t row = crow[c];
        const int64_t a = P_row[row] + cstart[c], b = min(a + kChunk, P_row[row + 1]);
        const float2 yi = Y[row];
        float2 acc = make_float2(0.f, 0.f);
        // kChunkBatch entries per lane at a time: the column and value loads,
        // then the gathers, all issued before any is used
        for (int64_t e0 = a + lane; e0 < b; e0 += 32 * kChunkBatch) {
            int cc[kChunkBatch];
            float pv[kChunkBatch];
#pragma unroll
            for (int t = 0; t < kChunkBatch; ++t) {
                const int64_t e = e0 + 32 * t;
                const bool ok = e < b;
                cc[t] = ok ? (D16 ? row + (int)P_d16[e] : P_col[e]) : row;
                pv[t] = ok ? __ldg(P_val + e) : 0.f;
            }
            float2 q[kChunkBatch];
#pragma unroll
            for (int t = 0; t < kChunkBatch; ++t) q[t] = __ldg(Y + min((unsigned)cc[t], (unsigned)(n - 1)));
#pragma unroll
            for (int t = 0; t < kChunkBatch; ++t) {
                const float2 d = sub_x2(yi, q[t]);
                const float w = pv[t] * rcp_approx(__fmaf_rn(d.y, d.y, __fmaf_rn(d.x, d.x, 1.0f)));
                acc = fma_x2(w, d, acc);
            }
        }
        const float ax = warp_sum(acc.x), ay = warp_sum(acc.y);
        if (lane == 0) partial[c] = make_float2(ax, ay);
    }
}

template <bool D16>
__global__ void __launch_bounds__(256) k_attr_chunks(const int64_t* __restrict__ P_row,
                                                     const int32_t* __restrict__ P_col,
                                                     const int16_t* __restrict__ P_d16,
                                                     const float* __restrict__ P_val, int32_t n,
                                                     const float2* __restrict__ Y, const int32_t* __restrict__ crow,
                                                     const int64_t* __restrict__ cstart, int32_t nchunks,
                                                     float2* __restrict__ partial)
{
    k_attr_chunks_body<D16>(P_row, P_col, P_d16, P_val, n, Y, crow, cstart, nchunks, partial);
}

// The long rows' chunk sums of every graph of a batch (graph = blockIdx.y).
template <bool D16>
__global__ void __launch_bounds__(256) k_attr_chunks_b(const BatchGraph* __restrict__ bg, int parity)
{
    const BatchGraph& b = bg[blockIdx.y];
    if (b.nchunks == 0) return;
    k_attr_chunks_body<D16>(b.P_row, b.P_col, b.P_d16, b.P_val, b.n, parity ? b.w.yalt : b.Y, b.crow, b.cstart,
                            b.nchunks, b.hpartial);
}

// Chunks per row (0 for rows of at most kHeavyRow entries).
__global__ void k_heavy_count(const int64_t* __restrict__ P_row, int32_t n, uint32_t* __restrict__ nch)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = P_row[i + 1] - P_row[i];
        nch[i] = len > kHeavyRow ? (uint32_t)((len + kChunk - 1) / kChunk) : 0u;
    }
}

// The chunk list of the long rows, their first chunks at base[row]; a
// chunk's start is its offset in the row, so the list serves both the CSR
// layout and the packed one (a chunk of kChunk entries covers whole 32-entry
// blocks of a packed row: the same entries as in CSR order).
__global__ void k_heavy_emit(const int64_t* __restrict__ P_row, int32_t n, const uint32_t* __restrict__ nch,
                             const uint32_t* __restrict__ base, int32_t* __restrict__ crow,
                             int64_t* __restrict__ cstart)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t m = nch[i];
        for (uint32_t c = 0; c < m; ++c) {
            crow[base[i] + c] = (int32_t)i;
            cstart[base[i] + c] = (int64_t)c * kChunk;
        }
    }
}

// Packed layout of the library's own P for the point phase: every row padded
// to a multiple of 4 entries (column offset 0, weight 0) and, inside each
// block of 32 entries of a row (the last block: s = 4m entries), entry
// t = a + m q (a < m, q < 4) of the block stored at slot 4 a + q.  A lane
// that loads slots 4a .. 4a+3 of a block as one vector then holds entries
// a, a + m, a + 2m, a + 3m, so the 8 lanes of a row gather the neighbours of
// m consecutive (sorted) columns at a time: after the breadth-first
// renumbering these lie close together, and each gather instruction touches
// fewer cache lines.  Columns are int16 offsets from the row; `far` is set if
// one does not fit, or a column is outside [0, n) or on the diagonal (the
// CSR arrays with int32 columns, whose gathers are clamped, are used then).
// Q_row[i] = P_row[i] + pads of the rows before i.
__global__ void k_pad_count(const int64_t* __restrict__ P_row, int32_t n, uint32_t* __restrict__ pads)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pads[i] = (uint32_t)((-(P_row[i + 1] - P_row[i])) & 3);
}

__global__ void k_pad_rows(const int64_t* __restrict__ P_row, int32_t n, const uint32_t* __restrict__ pads,
                           const uint32_t* __restrict__ pad_before, int64_t* __restrict__ Q_row)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Q_row[i] = P_row[i] + pad_before[i];
        if (i == n - 1) Q_row[n] = P_row[n] + pad_before[i] + pads[i];
    }
}

// C32: int32 columns (pads: the row itself, weight 0); `far` is set only
// for a column outside [0, n).  Else int16 offsets (pads: offset 0), `far`
// set also for an offset outside the int16 range or on the diagonal.
template <bool C32>
__global__ void k_pack_rows(const int64_t* __restrict__ P_row, const int32_t* __restrict__ P_col,
                            const float* __restrict__ P_val, int32_t n, const int64_t* __restrict__ Q_row,
                            void* __restrict__ Q_col, float* __restrict__ Q_val, int32_t* __restrict__ far)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
        const int64_t p0 = P_row[row], len = P_row[row + 1] - p0;
        const int64_t q0 = Q_row[row], lp = Q_row[row + 1] - q0;
        bool bad = false;
        for (int64_t t = lane; t < lp; t += 32) {
            const int64_t blk = t & ~(int64_t)31;
            const int m = (int)(min(lp - blk, (int64_t)32) >> 2);
            const int r = (int)(t - blk), a = r % m, q = r / m;
            int32_t c = C32 ? (int32_t)row : 0;
            float v = 0.f;
            if (t < len) {
                const int32_t col = P_col[p0 + t];
                const int64_t off = (int64_t)col - row;
                bad |= col < 0 || col >= n;
                if (!C32) bad |= off < -32767 || off > 32767 || off == 0;
                c = C32 ? col : (int32_t)off;
                v = P_val[p0 + t];
            }
            const int64_t dst = q0 + blk + 4 * a + q;
            if (C32) ((int32_t*)Q_col)[dst] = c;
            else ((int16_t*)Q_col)[dst] = (int16_t)c;
            Q_val[dst] = v;
        }
        if (__any_sync(FULL, bad) && lane == 0) atomicExch(far, 1);
    }
}

// The cost (Eq. 1 in the entropy reading) at Y: the sparse sums over P,
//   sum p ln p, sum p ln(1 + d^2) (KL with q_ij = (1+d^2)^-1 / Z, Eq. 4),
// the compression sum |X|^2, and optionally dC/dp_e = l_KL (ln p_e + 1 +
// ln(1 + d_e^2) + ln Z) for every stored entry.  Z, S and the entropy grid sum
// come from the grid phase.  One thread per row; FP64 sums per block, then
// the last block to finish combines them in block order (deterministic).
constexpr int kCostThreads = 256;
constexpr int kCostBlocks = 304;

__global__ void __launch_bounds__(kCostThreads) k_cost(const int64_t* __restrict__ P_row,
                                                       const int32_t* __restrict__ P_col,
                                                       const float* __restrict__ P_val, int32_t n,
                                                       const float2* __restrict__ Y, GridDev* G, float lam_kl,
                                                       float lam_c, float lam_r, float eps,
                                                       float* __restrict__ dP, double* __restrict__ blk,
                                                       double* __restrict__ cost)
{
    __shared__ double red[3][kCostThreads];
    __shared__ bool last;
    const float lnZ = (float)log(G->Z);
    double plogp = 0.0, plogk = 0.0, sq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 yi = Y[i];
        sq += (double)yi.x * yi.x + (double)yi.y * yi.y;
        const int64_t e1 = P_row[i + 1];
        for (int64_t e = P_row[i]; e < e1; ++e) {
            const float p = P_val[e];
            const int c = P_col[e];
            const unsigned cc = min((unsigned)c, (unsigned)(n - 1));
            const float2 yj = Y[cc];
            const float dx = yi.x - yj.x, dy = yi.y - yj.y;
            const float lk = log1pf(__fmaf_rn(dy, dy, dx * dx));
            if (p > 0.f) plogp += (double)p * (double)logf(p);
            plogk += (double)p * (double)lk;
            if (dP) dP[e] = lam_kl * (logf(p) + 1.0f + lk + lnZ);
        }
    }
    red[0][threadIdx.x] = plogp;
    red[1][threadIdx.x] = plogk;
    red[2][threadIdx.x] = sq;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) blk[3 * blockIdx.x + k] = red[k][0];
        __threadfence();
        last = atomicAdd(&G->ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < (int)gridDim.x; ++b)
        for (int k = 0; k < 3; ++k) t[k] += ((volatile double*)blk)[3 * b + k];
    G->ticket = 0;
    if (!cost) return;
    const double c_kl = (double)lam_kl * (t[0] + t[1] + G->S * log(G->Z));
    const double c_cmp = (double)lam_c / (2.0 * n) * t[2];
    const double c_ent = -(double)lam_r / (4.0 * (double)n * n) * (G->Lsum - (double)n * log((double)eps));
    cost[0] = c_kl;
    cost[1] = c_cmp;
    cost[2] = c_ent;
    cost[3] = c_kl + c_cmp + c_ent;
}

// Column range check of a caller-supplied P (the fused kernel only clamps).
__global__ void k_check_cols(const int64_t* __restrict__ P_row, const int32_t* __restrict__ P_col, int32_t n,
                             StatusBlock* status)
{
    const int64_t nnz = P_row[n];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = P_col[e];
        if ((unsigned)c >= (unsigned)n) record_error(status, LTSNET_ERR_BAD_GRAPH, c);
    }
}

cudaError_t launch_check_cols(const int64_t* P_row, const int32_t* P_col, int32_t n, StatusBlock* st, cudaStream_t s)
{
    k_check_cols<<<num_sms() * 8, 256, 0, s>>>(P_row, P_col, n, st);
    count_launches(1);
    return cudaGetLastError();
}

// ---- plain form ------------------------------------------------------------
template <int P>
__global__ void k_plain_gather(const float2* __restrict__ Y, int32_t n, const GridDev* __restrict__ G,
                               const float* __restrict__ fields, float* __restrict__ phi)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Sums F = gather_sums<P>(Y[i], G, fields);
        *(float4*)(phi + i * 8) = make_float4(F.R.x, F.R.y, F.E.x, F.E.y);
    }
}

__global__ void k_plain_attract(const int64_t* __restrict__ P_row, const int32_t* __restrict__ P_col,
                                const float* __restrict__ P_val, int32_t n, const float2* __restrict__ Y,
                                float2* __restrict__ attr, StatusBlock* status)
{
    const int lane = threadIdx.x & 31;
    const int64_t nnz = P_row[n];
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
         row += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const float2 yi = Y[row];
        const float2 a =
            warp_row_attraction(P_col, P_val, nnz, P_row[row], P_row[row + 1], yi.x, yi.y, Y, n, lane, status);
        if (lane == 0) attr[row] = a;
    }
}

template <bool UPDATE>
__global__ void k_plain_update(int32_t n, const float2* __restrict__ Y, float2* __restrict__ Ynew,
                               float2* __restrict__ upd, float2* __restrict__ gains, const GridDev* __restrict__ G,
                               const float* __restrict__ phi, const float2* __restrict__ attr, Stage st,
                               int32_t* __restrict__ bounds_next, float2* __restrict__ grad_out,
                               float* __restrict__ parts, StatusBlock* status)
{
    const Coeffs k = coeffs(G, st);
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = Y[i];
        Sums F;
        const float4 a = *(const float4*)(phi + i * 8);
        F.R = make_float2(a.x, a.y);
        F.E = make_float2(a.z, a.w);
        const PointOut o = point_gradient(p, attr[i], F, k);
        if (UPDATE) {
            float2 u = upd[i], gn = gains[i];
            const float2 yn = step(p, o.g, u, gn, st);
            upd[i] = u;
            gains[i] = gn;
            Ynew[i] = yn;
            if (!(isfinite(yn.x) && isfinite(yn.y))) record_error(status, LTSNET_ERR_NONFINITE, (int32_t)i);
            mn = fminf(mn, fminf(yn.x, yn.y));
            mx = fmaxf(mx, fmaxf(yn.x, yn.y));
        } else {
            grad_out[i] = o.g;
            if (!(isfinite(o.g.x) && isfinite(o.g.y))) record_error(status, LTSNET_ERR_NONFINITE, (int32_t)i);
            if (parts) {
                float* q = parts + i * 6;
                q[0] = o.A.x; q[1] = o.A.y; q[2] = o.R.x; q[3] = o.R.y; q[4] = o.E.x; q[5] = o.E.y;
            }
        }
    }
    if (UPDATE) block_bounds(mn, mx, bounds_next);
}

__global__ void k_terms(const GridDev* __restrict__ G, double* __restrict__ terms)
{
    terms[0] = G->Z;
    terms[1] = G->S;
    terms[2] = (double)G->I;
    terms[3] = (double)G->h;
    terms[4] = (double)G->lo;
    terms[5] = (double)G->c;
    terms[6] = (double)G->M;
    terms[7] = 0.0;
}

__global__ void k_init_state(float2* __restrict__ upd, float2* __restrict__ gains, int32_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        upd[i] = make_float2(0.f, 0.f);
        gains[i] = make_float2(1.f, 1.f);
    }
}

__global__ void k_count_unconverged(const uint8_t* __restrict__ conv, const int32_t* __restrict__ cnt, int32_t n,
                                    StatusBlock* st)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!conv[i] && cnt[i] > 0) atomicOr(&st->warn, 1);
}

int fused_blocks(int32_t n)
{
    const int64_t groups = ((int64_t)n + 31) / 32;
    const int64_t wpb = kFusedThreads / 32;
    int64_t b = (groups + wpb - 1) / wpb;
    const int64_t cap = (int64_t)num_sms() * 2;  // persistent: the blocks that fit at once
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

int flat_blocks(int64_t n, int per_sm = 8)
{
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <bool UPDATE>
cudaError_t launch_point_phase(const PStream& sp, int32_t n, const float2* Y, float2* Ynew, float2* upd,
                               float2* gains, const IterWs& w,
                               const IterShape& sh, const Stage& st, int parity, float2* grad, float* parts,
                               bool plain, cudaStream_t s)
{
    const int64_t* P_row = sp.row;
    const int32_t* P_col = sp.col;
    const int16_t* P_d16 = sp.d16;
    const float* P_val = sp.val;
    const HeavyRows& hr = sp.hr;
    int32_t* bn = w.bounds + 2 * (parity ^ 1);
    if (!plain && hr.nchunks > 0) {
        int64_t cb = ((int64_t)hr.nchunks * 32 + 255) / 256;
        if (cb > num_sms() * 8) cb = num_sms() * 8;
        if (sp.fmt == kFmtPk16)
            k_attr_chunks<true><<<(unsigned)cb, 256, 0, s>>>(P_row, P_col, P_d16, P_val, n, Y, hr.crow, hr.cstart,
                                                             hr.nchunks, hr.partial);
        else
            k_attr_chunks<false><<<(unsigned)cb, 256, 0, s>>>(P_row, P_col, P_d16, P_val, n, Y, hr.crow, hr.cstart,
                                                              hr.nchunks, hr.partial);
        count_launches(1);
    }
    profile_start(LTSNET_KERNEL_FUSED_UPDATE, s);
    if (!plain) {
        const int nb = fused_blocks(n);
#define LT_FUSED_F(PP, FF)                                                                                   \
    k_fused<PP, UPDATE, FF><<<nb, kFusedThreads, kFusedSmem, s>>>(P_row, P_col, P_d16, P_val, n, Y, Ynew, upd,  \
                                                                  gains, w.g, w.fields, st, bn, grad, parts,   \
                                                                  w.st, hr.hbase, hr.partial)
#define LT_FUSED(PP)                                                   \
    if (sp.fmt == kFmtPk16) LT_FUSED_F(PP, kFmtPk16);                  \
    else if (sp.fmt == kFmtPk32) LT_FUSED_F(PP, kFmtPk32);             \
    else LT_FUSED_F(PP, kFmtCsr)
        switch (sh.P) {
            case 2: LT_FUSED(2); break;
            case 3: LT_FUSED(3); break;
            case 4: LT_FUSED(4); break;
            default: LT_FUSED(5); break;
        }
#undef LT_FUSED
#undef LT_FUSED_F
        count_launches(1);
    } else {
        const int nb = flat_blocks(n);
        switch (sh.P) {
            case 2: k_plain_gather<2><<<nb, 256, 0, s>>>(Y, n, w.g, w.fields, w.phi); break;
            case 3: k_plain_gather<3><<<nb, 256, 0, s>>>(Y, n, w.g, w.fields, w.phi); break;
            case 4: k_plain_gather<4><<<nb, 256, 0, s>>>(Y, n, w.g, w.fields, w.phi); break;
            default: k_plain_gather<5><<<nb, 256, 0, s>>>(Y, n, w.g, w.fields, w.phi); break;
        }
        int64_t ab = ((int64_t)n + 7) / 8;
        if (ab > num_sms() * 16) ab = num_sms() * 16;
        if (ab < 1) ab = 1;
        k_plain_attract<<<(unsigned)ab, 256, 0, s>>>(P_row, P_col, P_val, n, Y, w.attr, w.st);
        k_plain_update<UPDATE><<<nb, 256, 0, s>>>(n, Y, Ynew, upd, gains, w.g, w.phi, w.attr, st, bn, grad, parts,
                                                  w.st);
        count_launches(3);
    }
    profile_stop(LTSNET_KERNEL_FUSED_UPDATE, s);
    return cudaGetLastError();
}

bool params_ok(const ltsnet_params* p)
{
    if (!p) return false;
    if (!(p->perplexity > 0.f) || !(p->eps > 0.f) || !(p->box_width_max > 0.f)) return false;
    if (p->nodes_per_box < 2 || p->nodes_per_box > 5) return false;
    if (p->min_boxes < 1 || p->max_boxes < p->min_boxes) return false;
    if ((int64_t)2 * p->nodes_per_box * p->max_boxes > kLMax) return false;
    if (p->n_stages < 1 || !p->stages) return false;
    if (p->conv_mode != LTSNET_CONV_FFT && p->conv_mode != LTSNET_CONV_DFT_GEMM) return false;
    if (p->conv_mode == LTSNET_CONV_DFT_GEMM && (p->flags & LTSNET_FLAG_PLAIN)) return false;
    for (int i = 0; i < p->n_stages; ++i)
        if (p->stages[i].iters < 0) return false;
    return true;
}

Stage make_stage(const ltsnet_stage& s, float lr, int32_t n)
{
    Stage st;
    st.a_att = (float)(4.0 * (double)s.lambda_kl * (double)s.exaggeration);
    st.a_rep = (float)(4.0 * (double)s.lambda_kl);
    st.a_cmp = (float)((double)s.lambda_c / (double)n);
    st.a_ent = (float)((double)s.lambda_r / ((double)n * (double)n));
    st.momentum = s.momentum;
    st.lr = lr;
    return st;
}

float learning_rate(const ltsnet_params* p, int32_t n)
{
    if (p->learning_rate > 0.f) return p->learning_rate;
    const float a = (float)n / 12.0f;
    return a > 200.f ? a : 200.f;
}

// Stage of global iteration t: walk the schedule; past its end, the last stage.
const ltsnet_stage& stage_at(const ltsnet_params* p, int64_t t)
{
    int64_t acc = 0;
    for (int i = 0; i < p->n_stages; ++i) {
        acc += p->stages[i].iters;
        if (t < acc) return p->stages[i];
    }
    return p->stages[p->n_stages - 1];
}

int64_t schedule_length(const ltsnet_params* p)
{
    int64_t acc = 0;
    for (int i = 0; i < p->n_stages; ++i) acc += p->stages[i].iters;
    return acc;
}

size_t iter_ws_bytes(int32_t n, const ltsnet_params* p)
{
    Carve c(nullptr, 0);
    iter_carve(c, iter_shape(n, p));
    return align_up(c.off, 256);
}

cudaError_t set_fused_attrs()
{
    cudaError_t e;
    const int fs = (int)kFusedSmem;
#define LT_ATTR(PP, UU, DD)                                                                                  \
    if ((e = cudaFuncSetAttribute(k_fused<PP, UU, DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, fs))) \
        return e;
    LT_ATTR(2, true, false) LT_ATTR(3, true, false) LT_ATTR(4, true, false) LT_ATTR(5, true, false)
    LT_ATTR(2, false, false) LT_ATTR(3, false, false) LT_ATTR(4, false, false) LT_ATTR(5, false, false)
    LT_ATTR(2, true, true) LT_ATTR(3, true, true) LT_ATTR(4, true, true) LT_ATTR(5, true, true)
    LT_ATTR(2, false, true) LT_ATTR(3, false, true) LT_ATTR(4, false, true) LT_ATTR(5, false, true)
#undef LT_ATTR
    return cudaSuccess;
}

// Every kernel's dynamic shared-memory limit is raised to the most any
// supported configuration asks for, once on each device that runs them.
cudaError_t ensure_attrs()
{
    cudaError_t e = once_per_device(kOnceGridAttrs, grid_set_smem_attrs);
    if (e != cudaSuccess) return e;
    if ((e = once_per_device(kOnceDft, dft_set_attrs)) != cudaSuccess) return e;
    return once_per_device(kOnceFusedAttrs, set_fused_attrs);
}

ltsnet_status read_status(StatusBlock* st, cudaStream_t s)
{
    StatusBlock h;
    LT_CUDA(cudaMemcpyAsync(&h, st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    if (h.code != 0) return (ltsnet_status)h.code;
    if (h.warn & 1) return LTSNET_WARN_NOT_CONVERGED;
    return LTSNET_OK;
}

// The loop over iterations [t0, t0 + niter) on a carved iteration workspace.
// One iteration i (local index; parity i & 1 picks the layout buffer and
// the bounds slot): grid phase, then the point phase.
cudaError_t one_iteration(const PStream& sp, int32_t n,
                          const ltsnet_params* p, float2* Y, float2* upd, float2* gains, const IterWs& w,
                          const IterShape& sh, const Stage& st, int parity, bool plain, cudaStream_t s)
{
    float2* cur = parity ? w.yalt : Y;
    float2* nxt = parity ? Y : w.yalt;
    cudaError_t e = launch_grid_phase(w, sh, p, cur, parity, plain, s);
    if (e != cudaSuccess) return e;
    return launch_point_phase<true>(sp, n, cur, nxt, upd, gains, w, sh, st, parity, nullptr, nullptr, plain, s);
}

bool same_stage(const ltsnet_stage& a, const ltsnet_stage& b)
{
    return a.lambda_kl == b.lambda_kl && a.lambda_c == b.lambda_c && a.lambda_r == b.lambda_r &&
           a.exaggeration == b.exaggeration && a.momentum == b.momentum;
}

// The loop over iterations [t0, t0 + niter).  Runs of iterations with the
// same stage are replayed from a CUDA graph holding two iterations (one per
// layout parity), captured on an internal stream and launched on `s`; the
// graph's launches are counted as their kernels.  While kernels are being
// timed one by one (ltsnet_profile_begin) every iteration is launched
// directly.
// sp is P in the format the point phase streams (CSR or a packed layout).
ltsnet_status optimize_core(const PStream& sp, int32_t n,
                            const ltsnet_params* p, float2* Y, float2* upd, float2* gains, int32_t t0, int32_t niter,
                            const IterWs& w, const IterShape& sh, cudaStream_t s)
{
    const bool plain = (p->flags & LTSNET_FLAG_PLAIN) != 0;
    const float lr = learning_rate(p, n);
    LT_CUDA(ensure_attrs());
    LT_CUDA(launch_psum(w, sp.row, n, sp.val, s));
    LT_CUDA(launch_bounds_init(w, Y, n, 0, s));
    AuxStreams* aux = nullptr;
    const bool graphs = !profiling_active() && aux_streams(&aux) == cudaSuccess;
    int32_t i = 0;
    while (i < niter) {
        const ltsnet_stage& sg = stage_at(p, (int64_t)t0 + i);
        int32_t run = 1;
        while (i + run < niter && same_stage(stage_at(p, (int64_t)t0 + i + run), sg)) ++run;
        const Stage st = make_stage(sg, lr, n);
        int32_t done = 0;
        if ((i & 1) && run > 0) {  // align to an even iteration
            LT_CUDA(one_iteration(sp, n, p, Y, upd, gains, w, sh, st, 1, plain, s));
            done = 1;
        }
        const int32_t pairs = graphs ? (run - done) / 2 : 0;
        if (pairs >= 2) {
            const int64_t c0 = thread_launch_count();
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            LT_CUDA(cudaStreamBeginCapture(aux->capture, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = one_iteration(sp, n, p, Y, upd, gains, w, sh, st, 0, plain, aux->capture);
            if (e == cudaSuccess)
                e = one_iteration(sp, n, p, Y, upd, gains, w, sh, st, 1, plain, aux->capture);
            cudaError_t e2 = cudaStreamEndCapture(aux->capture, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                LT_CUDA(e != cudaSuccess ? e : e2);
            }
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            LT_CUDA(e);
            const int64_t per = thread_launch_count() - c0;
            for (int32_t q = 0; q < pairs; ++q) {
                e = cudaGraphLaunch(exec, s);
                if (e != cudaSuccess) break;
            }
            cudaGraphExecDestroy(exec);  // freed once its launches complete
            LT_CUDA(e);
            count_launches(per * (pairs - 1));
            done += 2 * pairs;
        }
        for (; done < run; ++done)
            LT_CUDA(one_iteration(sp, n, p, Y, upd, gains, w, sh, st, (i + done) & 1, plain, s));
        i += run;
    }
    if (niter & 1) LT_CUDA(cudaMemcpyAsync(Y, w.yalt, sizeof(float2) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    return LTSNET_OK;
}

struct RunWs {
    StatusBlock* st;
    int32_t* nbr;
    uint16_t* hop;
    int32_t* cnt;
    double* beta;
    double* pcond;
    int64_t* Q_row;    // packed layout of P for the point phase (k_pack_rows), in
    int32_t* Q_col;    // the symmetrisation's scratch, dead once P is built
    float* Q_val;      // (int16 offsets or int32 columns in Q_col); null when
                       // it does not fit there (tiny graphs)
    int32_t* far;      // set when some |col - row| exceeds the int16 range
    uint32_t* hnch;    // chunks per long row of P
    uint32_t* hbase;   // first chunk of each long row
    uint32_t* htmp;    // scan scratch
    int32_t* hcrow;    // chunk -> row
    int64_t* hcstart;  // chunk -> first entry
    float2* hpartial;  // chunk sums
    int64_t hmax;      // chunk capacity
    uint8_t* conv;
    int64_t* P_row;
    int32_t* P_col;
    float* P_val;
    float2* upd;
    float2* gains;
    int64_t* row_ptr;  // host-input copies (ltsnet_run_host)
    int32_t* col;
    float2* Y;
    int32_t* order;    // breadth-first renumbering: order[new] = old, inv[old] = new
    int32_t* inv;
    int32_t* nbr2;     // conditional rows in the new numbering
    double* pcond2;
    int32_t* cnt2;
    float2* Y2;
    void* ord;
    size_t ord_bytes;
    void* sym;
    size_t sym_bytes;
    void* iter;
    size_t iter_bytes;
};

int32_t k_of(const ltsnet_params* p) { return (int32_t)ceil(3.0 * (double)p->perplexity - 1e-9); }

RunWs run_carve(Carve& c, int32_t n, int64_t m2, const ltsnet_params* p, bool host_inputs)
{
    RunWs r;
    const int32_t k = k_of(p);
    const int64_t nk = (int64_t)n * k;
    r.st = c.take<StatusBlock>(1);
    r.nbr = c.take<int32_t>(nk);
    r.hop = c.take<uint16_t>(nk);
    r.cnt = c.take<int32_t>(n);
    r.beta = c.take<double>(n);
    r.pcond = c.take<double>(nk);
    r.far = c.take<int32_t>(1);
    r.hnch = c.take<uint32_t>(n);
    r.hbase = c.take<uint32_t>(n);
    r.htmp = c.take<uint32_t>(scan_tmp_words(n));
    // chunks: at most 2 nnz / kChunk (each long row has more than kChunk
    // entries, and nnz <= 2 n k)
    r.hmax = 2 * (2 * nk) / kChunk + 1;
    r.hcrow = c.take<int32_t>(r.hmax);
    r.hcstart = c.take<int64_t>(r.hmax);
    r.hpartial = c.take<float2>(r.hmax);
    r.conv = c.take<uint8_t>(n);
    r.P_row = c.take<int64_t>((int64_t)n + 1);
    r.P_col = c.take<int32_t>(2 * nk);
    r.P_val = c.take<float>(2 * nk);
    r.upd = c.take<float2>(n);
    r.gains = c.take<float2>(n);
    r.row_ptr = host_inputs ? c.take<int64_t>((int64_t)n + 1) : nullptr;
    r.col = host_inputs ? c.take<int32_t>(m2) : nullptr;
    r.Y = host_inputs ? c.take<float2>(n) : nullptr;
    r.order = c.take<int32_t>(n);
    r.inv = c.take<int32_t>(n);
    r.nbr2 = c.take<int32_t>(nk);
    r.pcond2 = c.take<double>(nk);
    r.cnt2 = c.take<int32_t>(n);
    r.Y2 = c.take<float2>(n);
    r.ord_bytes = order_ws_bytes(n);
    r.ord = c.take<char>(r.ord_bytes);
    r.sym_bytes = ltsnet_symmetrize_workspace_size(n, k);
    r.sym = c.take<char>(r.sym_bytes);
    {
        // padded rows: at most nnz + 3 n <= 2 n k + 3 n entries
        const int64_t qcap = 2 * nk + 3 * (int64_t)n;
        Carve q(r.sym, r.sym_bytes);
        r.Q_row = q.take<int64_t>((int64_t)n + 1);
        r.Q_col = q.take<int32_t>(qcap);
        r.Q_val = q.take<float>(qcap);
        if (!q.ok()) r.Q_row = nullptr, r.Q_col = nullptr, r.Q_val = nullptr;
    }
    r.iter_bytes = iter_ws_bytes(n, p);
    r.iter = c.take<char>(r.iter_bytes);
    return r;
}

// P of a prepared run in the packed layout (Q_row already holds the padded
// row starts): int16 offsets (c32 false) or int32 columns; *fmt gets the
// format, or kFmtCsr when a column does not fit it (CSR is streamed then).
cudaError_t pack_rows(const RunWs& r, int32_t n, bool c32, cudaStream_t s, int* fmt)
{
    cudaError_t e = cudaMemsetAsync(r.far, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (c32)
        k_pack_rows<true><<<num_sms() * 8, 256, 0, s>>>(r.P_row, r.P_col, r.P_val, n, r.Q_row, r.Q_col, r.Q_val, r.far);
    else
        k_pack_rows<false><<<num_sms() * 8, 256, 0, s>>>(r.P_row, r.P_col, r.P_val, n, r.Q_row, r.Q_col, r.Q_val,
                                                         r.far);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int32_t far = 1;
    if ((e = cudaMemcpyAsync(&far, r.far, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *fmt = far != 0 ? kFmtCsr : (c32 ? kFmtPk32 : kFmtPk16);
    return cudaSuccess;
}

// The P a prepared run streams.
PStream stream_of(const RunWs& r, int fmt, const HeavyRows& hr)
{
    PStream sp;
    const bool pk = fmt != kFmtCsr;
    sp.row = pk ? r.Q_row : r.P_row;
    sp.col = fmt == kFmtPk32 ? r.Q_col : r.P_col;
    sp.d16 = fmt == kFmtPk16 ? (const int16_t*)r.Q_col : nullptr;
    sp.val = pk ? r.Q_val : r.P_val;
    sp.fmt = fmt;
    sp.hr = hr;
    return sp;
}

// C0 of one graph and the state the loop starts from: partial BFS,
// calibration, breadth-first renumbering, symmetrisation, the packed layout
// of P, long row chunks, update/gains.  *Yw gets the layout the loop works
// on (Y, or its renumbered copy in r.Y2).
struct Prepared {
    bool reordered = false;
    int fmt = kFmtCsr;  // kFmtPk16 / kFmtPk32: P packed (k_pack_rows) in Q_row / Q_col / Q_val
    HeavyRows hr;
    int64_t nnz = 0;
    float2* Yw = nullptr;
};

ltsnet_status run_prepare(const int64_t* row_ptr, const int32_t* col, int32_t n, const ltsnet_params* p, float2* Y,
                          const RunWs& r, cudaStream_t s, Prepared* out)
{
    const int32_t k = k_of(p);
    ltsnet_status rc = ltsnet_knn_bfs(row_ptr, col, n, k, r.nbr, r.hop, r.cnt, r.st, sizeof(StatusBlock), s);
    if (rc != LTSNET_OK) return rc;
    rc = ltsnet_calibrate(r.hop, r.cnt, n, k, p->perplexity, p->beta_tol, p->beta_max_steps, r.beta, r.pcond, r.conv,
                          s);
    if (rc != LTSNET_OK) return rc;
    k_count_unconverged<<<flat_blocks(n), 256, 0, s>>>(r.conv, r.cnt, n, r.st);
    count_launches(1);
    LT_CHECK_LAUNCH();
    // Breadth-first renumbering for locality of the neighbour gathers: the
    // conditional rows are relabelled before symmetrisation, so P is built
    // directly in the new numbering; the layout is permuted in and out.
    bool reordered = false;
    if (!(p->flags & LTSNET_FLAG_NO_REORDER)) LT_CUDA(bfs_order(row_ptr, col, n, r.order, r.inv, r.ord, s, &reordered));
    int64_t nnz = 0;
    if (reordered) {
        LT_CUDA(permute_conditional_rows(r.order, r.inv, r.nbr, r.pcond, r.cnt, n, k, r.nbr2, r.pcond2, r.cnt2, s));
        rc = ltsnet_symmetrize(r.nbr2, r.cnt2, r.pcond2, n, k, r.P_row, r.P_col, r.P_val, 2 * (int64_t)n * k, &nnz,
                               r.sym, r.sym_bytes, s);
    } else {
        rc = ltsnet_symmetrize(r.nbr, r.cnt, r.pcond, n, k, r.P_row, r.P_col, r.P_val, 2 * (int64_t)n * k, &nnz,
                               r.sym, r.sym_bytes, s);
    }
    if (rc != LTSNET_OK) return rc;
    // packed layout: int16 column offsets when every entry is within int16
    // range of its row, else int32 columns
    int fmt = kFmtCsr;
    if (!(p->flags & LTSNET_FLAG_PLAIN) && nnz > 0 && r.Q_row) {
        k_pad_count<<<flat_blocks(n), 256, 0, s>>>(r.P_row, n, r.hnch);
        LT_CUDA(scan_u32_exclusive(r.hnch, r.hbase, n, r.htmp, s));
        k_pad_rows<<<flat_blocks(n), 256, 0, s>>>(r.P_row, n, r.hnch, r.hbase, r.Q_row);
        count_launches(2);
        LT_CHECK_LAUNCH();
        LT_CUDA(pack_rows(r, n, false, s, &fmt));
        if (fmt == kFmtCsr) LT_CUDA(pack_rows(r, n, true, s, &fmt));
    }
    // rows of P too long for one 8-lane group: chunk lists
    HeavyRows hr;
    if (!(p->flags & LTSNET_FLAG_PLAIN) && nnz > 0) {
        k_heavy_count<<<flat_blocks(n), 256, 0, s>>>(r.P_row, n, r.hnch);
        count_launches(1);
        LT_CHECK_LAUNCH();
        LT_CUDA(scan_u32_exclusive(r.hnch, r.hbase, n, r.htmp, s));
        uint32_t last[2] = {0, 0};
        LT_CUDA(cudaMemcpyAsync(&last[0], r.hbase + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        LT_CUDA(cudaMemcpyAsync(&last[1], r.hnch + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        LT_CUDA(cudaStreamSynchronize(s));
        const int64_t nch = (int64_t)last[0] + last[1];
        if (nch > r.hmax) return LTSNET_ERR_WORKSPACE;
        if (nch > 0) {
            k_heavy_emit<<<flat_blocks(n), 256, 0, s>>>(r.P_row, n, r.hnch, r.hbase, r.hcrow, r.hcstart);
            count_launches(1);
            LT_CHECK_LAUNCH();
            hr.hbase = (const int32_t*)r.hbase;
            hr.crow = r.hcrow;
            hr.cstart = r.hcstart;
            hr.partial = r.hpartial;
            hr.nchunks = (int32_t)nch;
        }
    }
    k_init_state<<<flat_blocks(n), 256, 0, s>>>(r.upd, r.gains, n);
    count_launches(1);
    LT_CHECK_LAUNCH();
    float2* Yw = Y;
    if (reordered) {
        LT_CUDA(gather_rows2(Y, r.order, n, r.Y2, s));
        Yw = r.Y2;
    }
    out->reordered = reordered;
    out->fmt = fmt;
    out->hr = hr;
    out->nnz = nnz;
    out->Yw = Yw;
    return LTSNET_OK;
}

// After the loop: the layout back in the input's numbering, and the first
// error (or warning) recorded by the loop's or by C0's kernels.
ltsnet_status run_finish(int32_t n, float2* Y, const RunWs& r, const Prepared& pr, StatusBlock* iter_st,
                         cudaStream_t s)
{
    if (pr.reordered) LT_CUDA(gather_rows2(r.Y2, r.inv, n, Y, s));
    ltsnet_status a = read_status(iter_st, s);
    ltsnet_status b = read_status(r.st, s);
    if (a < 0) return a;
    return b;
}

ltsnet_status run_core(const int64_t* row_ptr, const int32_t* col, int32_t n, const ltsnet_params* p, float2* Y,
                       const RunWs& r, cudaStream_t s)
{
    Prepared pr;
    ltsnet_status rc = run_prepare(row_ptr, col, n, p, Y, r, s, &pr);
    if (rc != LTSNET_OK) return rc;
    const IterShape sh = iter_shape(n, p);
    Carve ic(r.iter, r.iter_bytes);
    const IterWs w = iter_carve(ic, sh);
    LT_CUDA(iter_reset(w, sh, s));
    const int64_t total = schedule_length(p);
    rc = optimize_core(stream_of(r, pr.fmt, pr.hr), n, p, pr.Yw, r.upd, r.gains, 0,
                       (int32_t)total, w, sh, s);
    if (rc != LTSNET_OK) return rc;
    return run_finish(n, Y, r, pr, w.st, s);
}

// The descent loop of a whole batch, one launch per phase over all graphs
// (ltsnet_run_batched's one-launch mode): the same kernels, order, stage
// runs and two-iteration CUDA graphs as optimize_core, every launch covering
// every graph (grid.y = graph).  bg[st] is the device descriptor array of
// schedule stage st; hg the host copy of stage 0's (for the per-graph
// start and end steps).
ltsnet_status batched_loop(BatchGraph* const* bg, const std::vector<BatchGraph>& hg, const BatchShape& bs,
                           const IterShape& sh, const ltsnet_params* p, int fmt, cudaStream_t s)
{
    const int32_t ng = (int32_t)hg.size();
    LT_CUDA(ensure_attrs());
    for (const BatchGraph& b : hg) {
        LT_CUDA(launch_psum(b.w, b.P_row, b.n, b.P_val, s));
        LT_CUDA(launch_bounds_init(b.w, b.Y, b.n, 0, s));
    }
    AuxStreams* aux = nullptr;
    const bool graphs = !profiling_active() && aux_streams(&aux) == cudaSuccess;
    const unsigned fblocks = (unsigned)std::max<int64_t>(1, ((int64_t)bs.max_n + kFusedWarps * 32 - 1) / (kFusedWarps * 32));
    int64_t max_chunks = 0;
    for (const BatchGraph& b : hg) max_chunks = std::max<int64_t>(max_chunks, b.nchunks);
    const unsigned cblocks = (unsigned)std::min<int64_t>(num_sms() * 2, (max_chunks * 32 + 255) / 256);
    auto iteration = [&](const BatchGraph* dbg, int parity, cudaStream_t st) -> cudaError_t {
        cudaError_t e = launch_grid_phase_batched(dbg, ng, bs, sh, p, parity, st);
        if (e != cudaSuccess) return e;
        if (max_chunks > 0) {
            // chunk sums of the long rows (graphs without any return at once)
            if (fmt == kFmtPk16) k_attr_chunks_b<true><<<dim3(cblocks, (unsigned)ng), 256, 0, st>>>(dbg, parity);
            else k_attr_chunks_b<false><<<dim3(cblocks, (unsigned)ng), 256, 0, st>>>(dbg, parity);
            count_launches(1);
        }
        profile_start(LTSNET_KERNEL_FUSED_UPDATE, st);
        const dim3 grid(fblocks, (unsigned)ng);
#define LT_FB(PP)                                                                                   \
    if (fmt == kFmtPk16) k_fused_b<PP, kFmtPk16><<<grid, kFusedThreads, kFusedSmem, st>>>(dbg, parity);    \
    else if (fmt == kFmtPk32) k_fused_b<PP, kFmtPk32><<<grid, kFusedThreads, kFusedSmem, st>>>(dbg, parity); \
    else k_fused_b<PP, kFmtCsr><<<grid, kFusedThreads, kFusedSmem, st>>>(dbg, parity)
        switch (sh.P) {
            case 2: LT_FB(2); break;
            case 3: LT_FB(3); break;
            case 4: LT_FB(4); break;
            default: LT_FB(5); break;
        }
#undef LT_FB
        count_launches(1);
        profile_stop(LTSNET_KERNEL_FUSED_UPDATE, st);
        return cudaGetLastError();
    };
    const int64_t total = schedule_length(p);
    int64_t i = 0;
    int32_t sidx = 0;
    while (i < total) {
        // the schedule's stages in order; zero-length stages are skipped
        int64_t acc = 0;
        for (sidx = 0; sidx < p->n_stages; ++sidx) {
            acc += p->stages[sidx].iters;
            if (i < acc) break;
        }
        const int64_t run = acc - i;
        const BatchGraph* dbg = bg[sidx];
        int64_t done = 0;
        if ((i & 1) && run > 0) {
            LT_CUDA(iteration(dbg, 1, s));
            done = 1;
        }
        const int64_t pairs = graphs ? (run - done) / 2 : 0;
        if (pairs >= 2) {
            const int64_t c0 = thread_launch_count();
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            LT_CUDA(cudaStreamBeginCapture(aux->capture, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = iteration(dbg, 0, aux->capture);
            if (e == cudaSuccess) e = iteration(dbg, 1, aux->capture);
            cudaError_t e2 = cudaStreamEndCapture(aux->capture, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                LT_CUDA(e != cudaSuccess ? e : e2);
            }
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            LT_CUDA(e);
            const int64_t per = thread_launch_count() - c0;
            for (int64_t q = 0; q < pairs; ++q) {
                e = cudaGraphLaunch(exec, s);
                if (e != cudaSuccess) break;
            }
            cudaGraphExecDestroy(exec);
            LT_CUDA(e);
            count_launches(per * (pairs - 1));
            done += 2 * pairs;
        }
        for (; done < run; ++done) LT_CUDA(iteration(dbg, (int)((i + done) & 1), s));
        i += run;
    }
    if (total & 1)
        for (const BatchGraph& b : hg)
            LT_CUDA(cudaMemcpyAsync(b.Y, b.w.yalt, sizeof(float2) * (size_t)b.n, cudaMemcpyDeviceToDevice, s));
    return LTSNET_OK;
}

}  // namespace
}  // namespace lt

using namespace lt;

extern "C" size_t ltsnet_gradient_workspace_size(int32_t n, const ltsnet_params* p)
{
    if (n < 0 || !params_ok(p)) return 0;
    return iter_ws_bytes(n, p);
}

extern "C" size_t ltsnet_optimize_workspace_size(int32_t n, const ltsnet_params* p)
{
    return ltsnet_gradient_workspace_size(n, p);
}

static bool aligned16(const void* a, const void* b, const void* c)
{
    return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) == 0;
}

static ltsnet_status prepare_iter(int32_t n, const ltsnet_params* p, void* ws, size_t ws_bytes, IterShape& sh,
                                  IterWs& w, cudaStream_t s)
{
    if ((uintptr_t)ws & 255) return LTSNET_ERR_WORKSPACE;
    sh = iter_shape(n, p);
    Carve c(ws, ws_bytes);
    w = iter_carve(c, sh);
    if (!c.ok()) return LTSNET_ERR_WORKSPACE;
    LT_CUDA(iter_reset(w, sh, s));
    return LTSNET_OK;
}

extern "C" ltsnet_status ltsnet_gradient(const int64_t* P_row, const int32_t* P_col, const float* P_val, int32_t n,
                                         const float* Y, const ltsnet_stage* stage, const ltsnet_params* p,
                                         float* grad, float* parts, double* terms, void* ws, size_t ws_bytes,
                                         ltsnet_stream stream)
{
    if (n < 1 || !P_row || !P_col || !P_val || !Y || !stage || !grad || !ws || !params_ok(p))
        return LTSNET_ERR_INVALID_ARG;
    if (!aligned16(P_col, P_val, Y) || ((uintptr_t)grad & 7)) return LTSNET_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    IterShape sh;
    IterWs w;
    ltsnet_status rc = prepare_iter(n, p, ws, ws_bytes, sh, w, s);
    if (rc != LTSNET_OK) return rc;
    LT_CUDA(ensure_attrs());
    const bool plain = (p->flags & LTSNET_FLAG_PLAIN) != 0;
    const Stage st = make_stage(*stage, learning_rate(p, n), n);
    LT_CUDA(launch_check_cols(P_row, P_col, n, w.st, s));
    LT_CUDA(launch_psum(w, P_row, n, P_val, s));
    LT_CUDA(launch_bounds_init(w, (const float2*)Y, n, 0, s));
    LT_CUDA(launch_grid_phase(w, sh, p, (const float2*)Y, 0, plain, s));
    LT_CUDA(launch_point_phase<false>(csr_stream(P_row, P_col, P_val), n, (const float2*)Y, nullptr, nullptr, nullptr,
                                      w, sh, st, 0, (float2*)grad, parts, plain, s));
    if (terms) {
        k_terms<<<1, 1, 0, s>>>(w.g, terms);
        count_launches(1);
        LT_CHECK_LAUNCH();
    }
    return LTSNET_OK;
}

extern "C" ltsnet_status ltsnet_cost(const int64_t* P_row, const int32_t* P_col, const float* P_val, int32_t n,
                                     const float* Y, const ltsnet_stage* stage, const ltsnet_params* p, double* cost,
                                     float* dC_dPval, void* ws, size_t ws_bytes, ltsnet_stream stream)
{
    if (n < 1 || !P_row || !P_col || !P_val || !Y || !stage || (!cost && !dC_dPval) || !ws || !params_ok(p))
        return LTSNET_ERR_INVALID_ARG;
    if (!aligned16(P_col, P_val, Y) || ((uintptr_t)cost & 7) || ((uintptr_t)dC_dPval & 3))
        return LTSNET_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    IterShape sh;
    IterWs w;
    ltsnet_status rc = prepare_iter(n, p, ws, ws_bytes, sh, w, s);
    if (rc != LTSNET_OK) return rc;
    LT_CUDA(ensure_attrs());
    const bool plain = (p->flags & LTSNET_FLAG_PLAIN) != 0;
    LT_CUDA(launch_check_cols(P_row, P_col, n, w.st, s));
    LT_CUDA(launch_psum(w, P_row, n, P_val, s));
    LT_CUDA(launch_bounds_init(w, (const float2*)Y, n, 0, s));
    LT_CUDA(launch_grid_phase(w, sh, p, (const float2*)Y, 0, plain, s));
    LT_CUDA(cudaMemsetAsync(&w.g->ticket, 0, sizeof(int32_t), s));
    k_cost<<<kCostBlocks, kCostThreads, 0, s>>>(P_row, P_col, P_val, n, (const float2*)Y, w.g, stage->lambda_kl,
                                                stage->lambda_c, stage->lambda_r, p->eps, dC_dPval, w.sblk, cost);
    count_launches(1);
    LT_CHECK_LAUNCH();
    return LTSNET_OK;
}

extern "C" ltsnet_status ltsnet_grad_pvals(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                                           int32_t n, const float* Y, const ltsnet_stage* stage,
                                           const ltsnet_params* p, float* dC_dPval, void* ws, size_t ws_bytes,
                                           ltsnet_stream stream)
{
    if (!dC_dPval) return LTSNET_ERR_INVALID_ARG;
    return ltsnet_cost(P_row, P_col, P_val, n, Y, stage, p, nullptr, dC_dPval, ws, ws_bytes, stream);
}

extern "C" ltsnet_status ltsnet_optimize(const int64_t* P_row, const int32_t* P_col, const float* P_val, int32_t n,
                                         const ltsnet_params* p, float* Y, float* update, float* gains,
                                         int32_t start_iter, int32_t n_iter, void* ws, size_t ws_bytes,
                                         ltsnet_stream stream)
{
    if (n < 1 || !P_row || !P_col || !P_val || !Y || !update || !gains || !ws || !params_ok(p) || start_iter < 0 ||
        n_iter < 0)
        return LTSNET_ERR_INVALID_ARG;
    if (!aligned16(P_col, P_val, Y) || (((uintptr_t)update | (uintptr_t)gains) & 7)) return LTSNET_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    IterShape sh;
    IterWs w;
    ltsnet_status rc = prepare_iter(n, p, ws, ws_bytes, sh, w, s);
    if (rc != LTSNET_OK) return rc;
    LT_CUDA(launch_check_cols(P_row, P_col, n, w.st, s));
    return optimize_core(csr_stream(P_row, P_col, P_val), n, p, (float2*)Y, (float2*)update, (float2*)gains,
                         start_iter, n_iter, w, sh, s);
}

extern "C" size_t ltsnet_run_workspace_size(int32_t n, int64_t nnz_graph, const ltsnet_params* p)
{
    if (n < 1 || nnz_graph < 0 || !params_ok(p)) return 0;
    Carve c(nullptr, 0);
    run_carve(c, n, nnz_graph, p, true);
    return align_up(c.off, 256);
}

extern "C" ltsnet_status ltsnet_run(const int64_t* row_ptr, const int32_t* col, int32_t n, const ltsnet_params* p,
                                    float* Y, void* ws, size_t ws_bytes, ltsnet_stream stream)
{
    if (n < 1 || !row_ptr || !col || !Y || !ws || !params_ok(p)) return LTSNET_ERR_INVALID_ARG;
    if (k_of(p) > LTSNET_MAX_K) return LTSNET_ERR_INVALID_ARG;
    if ((uintptr_t)ws & 255) return LTSNET_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Carve c(ws, ws_bytes);
    RunWs r = run_carve(c, n, 0, p, false);
    if (!c.ok()) return LTSNET_ERR_WORKSPACE;
    LT_CUDA(cudaMemsetAsync(r.st, 0, sizeof(StatusBlock), s));
    return run_core(row_ptr, col, n, p, (float2*)Y, r, s);
}

// ---- many independent graphs -------------------------------------------
// Graph g occupies vertices [vtx_off[g], vtx_off[g+1]) of Y, its CSR row
// pointers row_ptr[vtx_off[g] + g .. vtx_off[g+1] + g] (local, from 0) and its
// columns col[edge_off[g] .. edge_off[g+1]) (local ids).  Host worker threads,
// each with its own stream and workspace slice, take the graphs largest first
// and run the whole method on each; graphs share nothing, so each result is
// the one ltsnet_run gives for that graph alone.

static bool batch_ok(int32_t n_graphs, const int64_t* vtx_off, const int64_t* edge_off, int64_t& max_n,
                     int64_t& max_m)
{
    if (n_graphs < 1 || !vtx_off || !edge_off || vtx_off[0] != 0 || edge_off[0] != 0) return false;
    max_n = 0;
    max_m = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        const int64_t ng = vtx_off[g + 1] - vtx_off[g], mg = edge_off[g + 1] - edge_off[g];
        if (ng < 1 || ng > INT32_MAX || mg < 0) return false;
        max_n = std::max(max_n, ng);
        max_m = std::max(max_m, mg);
    }
    return true;
}

// The parameters graph g of a batch runs with: p, with the graph's own grid
// cap where cfg->max_boxes gives one.
static ltsnet_params graph_params(const ltsnet_params* p, const ltsnet_batch_config* cfg, int32_t g)
{
    ltsnet_params q = *p;
    if (cfg->max_boxes && cfg->max_boxes[g] > 0) q.max_boxes = cfg->max_boxes[g];
    return q;
}

static bool batch_cfg_ok(const ltsnet_batch_config* cfg)
{
    return cfg && (cfg->mode == LTSNET_BATCH_ONE_LAUNCH || cfg->mode == LTSNET_BATCH_PER_GRAPH) &&
           cfg->n_workers >= 1 && cfg->n_workers <= 64 && cfg->fft_blocks >= 0 && cfg->fft_blocks <= 64 &&
           cfg->spread_blocks >= 0 && cfg->spread_blocks <= 64;
}

// Every graph's parameters are valid (the per-graph caps included).
static bool batch_params_ok(int32_t n_graphs, const ltsnet_params* p, const ltsnet_batch_config* cfg)
{
    for (int32_t g = 0; g < n_graphs; ++g) {
        const ltsnet_params q = graph_params(p, cfg, g);
        if (!params_ok(&q)) return false;
    }
    return true;
}

// Workspace of the one-launch mode: a run workspace per graph (C0, P, state,
// iteration workspace, sized for the graph's own grid cap), then one
// descriptor array per schedule stage.
static size_t one_launch_slices(int32_t n_graphs, const int64_t* vtx_off, const int64_t* edge_off,
                                const ltsnet_params* p, const ltsnet_batch_config* cfg, std::vector<size_t>* offs)
{
    size_t off = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        const ltsnet_params q = graph_params(p, cfg, g);
        const size_t one = ltsnet_run_workspace_size((int32_t)(vtx_off[g + 1] - vtx_off[g]),
                                                     edge_off[g + 1] - edge_off[g], &q);
        if (one == 0) return 0;
        if (offs) offs->push_back(off);
        off += align_up(one, 256);
    }
    return off + align_up(sizeof(BatchGraph) * (size_t)n_graphs, 256) * (size_t)p->n_stages;
}

// Slice of one worker in the per-graph mode: the largest run workspace of
// any graph of the batch.
static size_t per_graph_slice(int32_t n_graphs, const int64_t* vtx_off, const int64_t* edge_off,
                              const ltsnet_params* p, const ltsnet_batch_config* cfg)
{
    size_t slice = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        const ltsnet_params q = graph_params(p, cfg, g);
        const size_t one = ltsnet_run_workspace_size((int32_t)(vtx_off[g + 1] - vtx_off[g]),
                                                     edge_off[g + 1] - edge_off[g], &q);
        if (one == 0) return 0;
        slice = std::max(slice, align_up(one, 256));
    }
    return slice;
}

extern "C" size_t ltsnet_run_batched_workspace_size(int32_t n_graphs, const int64_t* vtx_off,
                                                    const int64_t* edge_off, const ltsnet_params* p,
                                                    const ltsnet_batch_config* cfg)
{
    int64_t max_n, max_m;
    if (!params_ok(p) || !batch_cfg_ok(cfg) || !batch_ok(n_graphs, vtx_off, edge_off, max_n, max_m)) return 0;
    if (!batch_params_ok(n_graphs, p, cfg)) return 0;
    if (cfg->mode == LTSNET_BATCH_ONE_LAUNCH) return one_launch_slices(n_graphs, vtx_off, edge_off, p, cfg, nullptr);
    const size_t one = per_graph_slice(n_graphs, vtx_off, edge_off, p, cfg);
    if (one == 0) return 0;
    return one * (size_t)std::min(cfg->n_workers, n_graphs);
}

extern "C" ltsnet_status ltsnet_run_batched(int32_t n_graphs, const int64_t* vtx_off, const int64_t* edge_off,
                                            const int64_t* row_ptr, const int32_t* col, const ltsnet_params* p,
                                            float* Y, void* ws, size_t ws_bytes, const ltsnet_batch_config* cfg,
                                            ltsnet_stream stream)
{
    int64_t max_n, max_m;
    if (!row_ptr || !col || !Y || !ws || !params_ok(p) || !batch_cfg_ok(cfg)) return LTSNET_ERR_INVALID_ARG;
    if (!batch_ok(n_graphs, vtx_off, edge_off, max_n, max_m)) return LTSNET_ERR_INVALID_ARG;
    if (!batch_params_ok(n_graphs, p, cfg)) return LTSNET_ERR_INVALID_ARG;
    if (k_of(p) > LTSNET_MAX_K) return LTSNET_ERR_INVALID_ARG;
    if ((uintptr_t)ws & 255) return LTSNET_ERR_WORKSPACE;
    const bool one = cfg->mode == LTSNET_BATCH_ONE_LAUNCH;
    if (one && ((p->flags & LTSNET_FLAG_PLAIN) || p->conv_mode != LTSNET_CONV_FFT)) return LTSNET_ERR_INVALID_ARG;
    const int32_t workers = std::min(cfg->n_workers, n_graphs);
    std::vector<size_t> offs;
    size_t slice = 0;
    if (one) {
        const size_t need = one_launch_slices(n_graphs, vtx_off, edge_off, p, cfg, &offs);
        if (need == 0 || ws_bytes < need) return LTSNET_ERR_WORKSPACE;
    } else {
        slice = per_graph_slice(n_graphs, vtx_off, edge_off, p, cfg);
        if (slice == 0 || ws_bytes < slice * (size_t)workers) return LTSNET_ERR_WORKSPACE;
    }
    int dev = 0;
    LT_CUDA(cudaGetDevice(&dev));
    // inputs written on the caller's stream are visible to the workers
    LT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<int32_t> order(n_graphs);
    for (int32_t g = 0; g < n_graphs; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return vtx_off[a + 1] - vtx_off[a] > vtx_off[b + 1] - vtx_off[b];
    });
    std::atomic<int32_t> next{0};
    std::atomic<int> first_err{0};
    // keeps the first error; a warning only while there is none
    auto note = [&](int rc) {
        int cur = first_err.load();
        while ((rc < 0 && cur >= 0) || (rc > 0 && cur == 0))
            if (first_err.compare_exchange_weak(cur, rc)) break;
    };
    std::vector<ltsnet_params> gp(n_graphs);
    for (int32_t g = 0; g < n_graphs; ++g) gp[g] = graph_params(p, cfg, g);
    auto carve_graph = [&](int32_t g, void* base, size_t bytes, RunWs* r) {
        Carve c(base, bytes);
        *r = run_carve(c, (int32_t)(vtx_off[g + 1] - vtx_off[g]), 0, &gp[g], false);
        return c.ok();
    };
    // per-graph mode: every graph through run_core on the workers; one-launch
    // mode: the workers run C0 of every graph into its own slice
    std::vector<Prepared> prep(one ? n_graphs : 0);
    auto work = [&](int32_t wi) {
        cudaStream_t s = nullptr;
        if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            note((int)LTSNET_ERR_CUDA);
            return;
        }
        for (int32_t t = next.fetch_add(1); t < n_graphs; t = next.fetch_add(1)) {
            const int32_t g = order[t];
            const int32_t ng = (int32_t)(vtx_off[g + 1] - vtx_off[g]);
            RunWs r;
            void* base = one ? (char*)ws + offs[g] : (char*)ws + slice * (size_t)wi;
            const size_t bytes =
                one ? align_up(ltsnet_run_workspace_size(ng, edge_off[g + 1] - edge_off[g], &gp[g]), 256) : slice;
            ltsnet_status rc = LTSNET_OK;
            if (!carve_graph(g, base, bytes, &r)) rc = LTSNET_ERR_WORKSPACE;
            else if (cudaMemsetAsync(r.st, 0, sizeof(StatusBlock), s) != cudaSuccess) rc = LTSNET_ERR_CUDA;
            else if (one)
                rc = run_prepare(row_ptr + vtx_off[g] + g, col + edge_off[g], ng, &gp[g], (float2*)Y + vtx_off[g], r,
                                 s, &prep[g]);
            else
                rc = run_core(row_ptr + vtx_off[g] + g, col + edge_off[g], ng, &gp[g], (float2*)Y + vtx_off[g], r, s);
            note(rc);
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int32_t wi = 1; wi < workers; ++wi) pool.emplace_back(work, wi);
    work(0);
    for (std::thread& t : pool) t.join();
    if (!one || first_err.load() < 0) {
        if (!one && cfg->max_boxes_used)
            for (int32_t g = 0; g < n_graphs; ++g) cfg->max_boxes_used[g] = -1;  // not tracked in this mode
        return (ltsnet_status)first_err.load();
    }
    // one launch per phase over all graphs
    cudaStream_t s = (cudaStream_t)stream;
    // one format for the whole batch: int16 packed if every graph's P fits
    // it, else int32 packed if every graph is packed (the int16 ones are
    // packed again with int32 columns below), else CSR
    int fmt = kFmtPk16;
    for (int32_t g = 0; g < n_graphs; ++g) {
        if (prep[g].fmt == kFmtCsr) fmt = kFmtCsr;
        else if (prep[g].fmt == kFmtPk32 && fmt == kFmtPk16) fmt = kFmtPk32;
    }
    ltsnet_params pmax = gp[0];  // the largest grid cap of the batch sizes the shared launch shapes
    for (int32_t g = 1; g < n_graphs; ++g) pmax.max_boxes = std::max(pmax.max_boxes, gp[g].max_boxes);
    const IterShape shmax = iter_shape((int32_t)max_n, &pmax);
    std::vector<BatchGraph> hg(n_graphs);
    std::vector<RunWs> rws(n_graphs);
    for (int32_t g = 0; g < n_graphs; ++g) {
        const int32_t ng = (int32_t)(vtx_off[g + 1] - vtx_off[g]);
        carve_graph(g, (char*)ws + offs[g],
                    align_up(ltsnet_run_workspace_size(ng, edge_off[g + 1] - edge_off[g], &gp[g]), 256), &rws[g]);
        const RunWs& r = rws[g];
        const IterShape sh = iter_shape(ng, &gp[g]);
        Carve ic(r.iter, r.iter_bytes);
        BatchGraph& b = hg[g];
        b.w = iter_carve(ic, sh);
        LT_CUDA(iter_reset(b.w, sh, s));
        if (fmt == kFmtPk32 && prep[g].fmt == kFmtPk16) {
            int f = kFmtCsr;
            LT_CUDA(pack_rows(r, ng, true, s, &f));
            if (f != kFmtPk32) return LTSNET_ERR_BAD_GRAPH;  // not reached: the int16 packing checked the columns
        }
        const PStream sp = stream_of(r, fmt, prep[g].hr);
        b.P_row = sp.row;
        b.P_col = sp.col;
        b.P_d16 = sp.d16;
        b.P_val = sp.val;
        b.Y = prep[g].Yw;
        b.upd = r.upd;
        b.gains = r.gains;
        b.n = ng;
        b.max_boxes = gp[g].max_boxes;
        const HeavyRows& hr = prep[g].hr;
        b.hbase = hr.hbase;
        b.crow = hr.crow;
        b.cstart = hr.cstart;
        b.hpartial = hr.partial;
        b.nchunks = hr.nchunks;
    }
    ltsnet_status rc = LTSNET_OK;
    {
        // descriptor arrays, one per schedule stage (the stage coefficients
        // depend on each graph's n)
        char* dbase = (char*)ws + one_launch_slices(n_graphs, vtx_off, edge_off, p, cfg, nullptr) -
                      align_up(sizeof(BatchGraph) * (size_t)n_graphs, 256) * (size_t)p->n_stages;
        std::vector<BatchGraph*> dbg(p->n_stages);
        for (int32_t st = 0; st < p->n_stages; ++st) {
            std::vector<BatchGraph> sg = hg;
            for (int32_t g = 0; g < n_graphs; ++g)
                sg[g].st = make_stage(p->stages[st], learning_rate(p, hg[g].n), hg[g].n);
            dbg[st] = (BatchGraph*)(dbase + align_up(sizeof(BatchGraph) * (size_t)n_graphs, 256) * (size_t)st);
            LT_CUDA(cudaMemcpyAsync(dbg[st], sg.data(), sizeof(BatchGraph) * (size_t)n_graphs, cudaMemcpyHostToDevice,
                                    s));
        }
        LT_CUDA(cudaStreamSynchronize(s));  // the host copies above are staged before they go out of scope
        BatchShape bs;
        bs.fft_blocks = cfg->fft_blocks > 0 ? cfg->fft_blocks : 4;
        bs.spread_blocks = cfg->spread_blocks > 0 ? cfg->spread_blocks : 8;
        bs.max_n = (int32_t)max_n;
        rc = batched_loop(dbg.data(), hg, bs, shmax, p, fmt, s);
    }
    if (rc != LTSNET_OK) return rc;
    for (int32_t g = 0; g < n_graphs; ++g) {
        if (cfg->max_boxes_used) {
            LT_CUDA(cudaMemcpyAsync(&cfg->max_boxes_used[g], &hg[g].w.g->imax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        }
        note(run_finish(hg[g].n, (float2*)Y + vtx_off[g], rws[g], prep[g], hg[g].w.st, s));
    }
    LT_CUDA(cudaStreamSynchronize(s));
    return (ltsnet_status)first_err.load();
}

extern "C" ltsnet_status ltsnet_run_host(const int64_t* row_ptr_host, const int32_t* col_host, int32_t n,
                                         const ltsnet_params* p, float* Y_host, void* ws, size_t ws_bytes,
                                         ltsnet_stream stream)
{
    if (n < 1 || !row_ptr_host || !col_host || !Y_host || !ws || !params_ok(p)) return LTSNET_ERR_INVALID_ARG;
    if (k_of(p) > LTSNET_MAX_K) return LTSNET_ERR_INVALID_ARG;
    if ((uintptr_t)ws & 255) return LTSNET_ERR_WORKSPACE;
    const int64_t m2 = row_ptr_host[n];
    if (m2 < 0) return LTSNET_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Carve c(ws, ws_bytes);
    RunWs r = run_carve(c, n, m2, p, true);
    if (!c.ok()) return LTSNET_ERR_WORKSPACE;
    LT_CUDA(cudaMemsetAsync(r.st, 0, sizeof(StatusBlock), s));
    LT_CUDA(cudaMemcpyAsync(r.row_ptr, row_ptr_host, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
    if (m2 > 0) LT_CUDA(cudaMemcpyAsync(r.col, col_host, sizeof(int32_t) * (size_t)m2, cudaMemcpyHostToDevice, s));
    LT_CUDA(cudaMemcpyAsync(r.Y, Y_host, sizeof(float2) * (size_t)n, cudaMemcpyHostToDevice, s));
    ltsnet_status rc = run_core(r.row_ptr, r.col, n, p, r.Y, r, s);
    if (rc < 0) return rc;
    LT_CUDA(cudaMemcpyAsync(Y_host, r.Y, sizeof(float2) * (size_t)n, cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    return rc;
}
