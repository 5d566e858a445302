// Quadtree (Barnes-Hut) gradient of BH-tsNET (Alg. 1) and FIt-tsNET
// (Alg. 2).  BH-tsNET takes the repulsive KL sums (C1) from the quadtree of
// BH-SNE and the entropy sum (C2) from the same tree (Eq. 7); FIt-tsNET
// takes C1 from the grid interpolation (ltsnet_gradient) and C2 from the
// tree.  The attraction is the exact sparse sum in both.
//
// The tree, identical to the oracle's so that both open the same nodes:
// - domain: the square at (min x, min y) of side e = the larger extent
//   (1 if both are 0), in FP32;
// - depth 16; a point's depth-16 column is min(65535, floor((x - lo) * s)),
//   s = 65536 / e, every FP32 operation rounded on its own; Morton code with
//   the column on the even bits; a depth-l node holds the points sharing
//   the code's top 2l bits, its cell width is e 2^-l; one-point nodes are
//   not split;
// - centres of mass from exact fixed point: q = rint((x - lo) 2^36 / e) in
//   FP64, summed as int64 (one exclusive scan over the code-sorted points,
//   a node's sum is a difference of two prefixes), then
//   c = lo + (sum q / |N|) (e 2^-36) in FP64, rounded to FP32; a one-point
//   node uses the point itself;
// - the summary test w_l^2 < theta^2 d^2 in FP32, every operation rounded
//   on its own; a node holding the point is always opened; an opened
//   depth-16 node contributes its points one by one.
//
// Build: bounds, codes, a stable radix sort by code (ids in the high word
// of the key keep equal codes in id order), the 64-bit prefix sums, then per
// depth a flag pass (a node starts where the code prefix changes inside an
// active parent), a scan (node ids), the nodes' ranges and centres, the
// parents' child links and the next depth's active flags.  Search: one
// thread per point in code order (neighbouring threads walk similar paths),
// an explicit stack, FP32 sums Zp, R, E per point; Z = sum Zp in FP64 in a
// fixed order.
#include <math.h>

#include <algorithm>

#include "prims.cuh"

namespace lt {
namespace {

constexpr int kQtThreads = 256;
constexpr int kQtLevels = 16;
constexpr int kQtStack = 64;  // > 3 * kQtLevels + 4
constexpr int kFixBits = 36;
constexpr int kQtBlocks = kSplitBlocks * 4;  // fixed: sizes workspace partials
constexpr int kScanChunk = 4096;  // int64 scan: elements per block

struct QtScal {
    int32_t lo_ord[2], hi_ord[2];
    float lo[2];
    float ext;
    float s;         // 65536 / ext
    double scale64;  // 2^36 / ext
    double step;     // ext 2^-36
    int32_t nn[kQtLevels + 1];  // nodes per depth
    int32_t pad[3];
};

__device__ __forceinline__ float sq_rn(float2 a, float2 b)
{
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

__global__ void k_qt_bounds(const float2* __restrict__ Y, int32_t n, QtScal* sc)
{
    float lx = INFINITY, ly = INFINITY, hx = -INFINITY, hy = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 y = Y[i];
        lx = fminf(lx, y.x);
        ly = fminf(ly, y.y);
        hx = fmaxf(hx, y.x);
        hy = fmaxf(hy, y.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(FULL, lx, o));
        ly = fminf(ly, __shfl_xor_sync(FULL, ly, o));
        hx = fmaxf(hx, __shfl_xor_sync(FULL, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(FULL, hy, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&sc->lo_ord[0], f2ord(lx));
        atomicMin(&sc->lo_ord[1], f2ord(ly));
        atomicMax(&sc->hi_ord[0], f2ord(hx));
        atomicMax(&sc->hi_ord[1], f2ord(hy));
    }
}

__global__ void k_qt_domain(QtScal* sc)
{
    const float lx = ord2f(sc->lo_ord[0]), ly = ord2f(sc->lo_ord[1]);
    float ext = fmaxf(__fsub_rn(ord2f(sc->hi_ord[0]), lx), __fsub_rn(ord2f(sc->hi_ord[1]), ly));
    if (!(ext > 0.0f)) ext = 1.0f;
    sc->lo[0] = lx;
    sc->lo[1] = ly;
    sc->ext = ext;
    sc->s = __fdiv_rn(65536.0f, ext);
    sc->scale64 = ldexp(1.0, kFixBits) / (double)ext;
    sc->step = (double)ext * ldexp(1.0, -kFixBits);
}

__device__ __forceinline__ uint32_t spread_bits(uint32_t v)  // 16 bits -> even bits of 32
{
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void k_qt_codes(const float2* __restrict__ Y, int32_t n, const QtScal* __restrict__ sc,
                           uint64_t* __restrict__ key)
{
    const float lx = sc->lo[0], ly = sc->lo[1], s = sc->s;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 y = Y[i];
        const uint32_t ix = (uint32_t)min(65535, (int)__fmul_rn(__fsub_rn(y.x, lx), s));
        const uint32_t iy = (uint32_t)min(65535, (int)__fmul_rn(__fsub_rn(y.y, ly), s));
        const uint32_t code = spread_bits(ix) | (spread_bits(iy) << 1);
        key[i] = ((uint64_t)i << 32) | code;
    }
}

// Sorted order: sid, the points, their codes and fixed-point offsets.
__global__ void k_qt_gather(const uint64_t* __restrict__ key, const float2* __restrict__ Y, int32_t n,
                            const QtScal* __restrict__ sc, int32_t* __restrict__ sid, float2* __restrict__ ys,
                            uint32_t* __restrict__ scode, long long* __restrict__ qx, long long* __restrict__ qy,
                            uint8_t* __restrict__ active)
{
    const double lx = (double)sc->lo[0], ly = (double)sc->lo[1], sc64 = sc->scale64;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[p];
        const int32_t i = (int32_t)(k >> 32);
        const float2 y = Y[i];
        sid[p] = i;
        ys[p] = y;
        scode[p] = (uint32_t)k;
        qx[p] = __double2ll_rn(__dmul_rn((double)y.x - lx, sc64));
        qy[p] = __double2ll_rn(__dmul_rn((double)y.y - ly, sc64));
        active[p] = n > 1;
    }
}

// Exclusive int64 scan of x and y together (prefix sums of the charges).
__global__ void __launch_bounds__(kQtThreads) k_scan64_reduce(const long long* __restrict__ a,
                                                              const long long* __restrict__ b, int32_t n,
                                                              long long* __restrict__ bs)
{
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    long long sa = 0, sb = 0;
    for (int64_t p = base + threadIdx.x; p < min((int64_t)n, base + kScanChunk); p += kQtThreads) {
        sa += a[p];
        sb += b[p];
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    __shared__ long long ra[kQtThreads / 32], rb[kQtThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        ra[threadIdx.x >> 5] = sa;
        rb[threadIdx.x >> 5] = sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kQtThreads / 32; ++q) {
            sa += ra[q];
            sb += rb[q];
        }
        bs[2 * blockIdx.x] = sa;
        bs[2 * blockIdx.x + 1] = sb;
    }
}

__global__ void k_scan64_top(long long* __restrict__ bs, int32_t nb)
{
    long long ra = 0, rb = 0;
    for (int q = 0; q < nb; ++q) {
        const long long a = bs[2 * q], b = bs[2 * q + 1];
        bs[2 * q] = ra;
        bs[2 * q + 1] = rb;
        ra += a;
        rb += b;
    }
}

// Each thread takes kScanChunk / kQtThreads consecutive elements.
__global__ void __launch_bounds__(kQtThreads) k_scan64_down(const long long* __restrict__ a,
                                                            const long long* __restrict__ b, int32_t n,
                                                            const long long* __restrict__ bs,
                                                            long long* __restrict__ pa, long long* __restrict__ pb)
{
    constexpr int per = kScanChunk / kQtThreads;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * per;
    long long ta = 0, tb = 0;
    for (int j = 0; j < per; ++j) {
        const int64_t p = base + j;
        if (p < n) {
            ta += a[p];
            tb += b[p];
        }
    }
    // exclusive scan of the thread totals across the block
    __shared__ long long sa[kQtThreads], sb[kQtThreads];
    sa[threadIdx.x] = ta;
    sb[threadIdx.x] = tb;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ra = bs[2 * blockIdx.x], rb = bs[2 * blockIdx.x + 1];
        for (int q = 0; q < kQtThreads; ++q) {
            const long long xa = sa[q], xb = sb[q];
            sa[q] = ra;
            sb[q] = rb;
            ra += xa;
            rb += xb;
        }
    }
    __syncthreads();
    long long ra = sa[threadIdx.x], rb = sb[threadIdx.x];
    for (int j = 0; j < per; ++j) {
        const int64_t p = base + j;
        if (p < n) {
            pa[p] = ra;
            pb[p] = rb;
            ra += a[p];
            rb += b[p];
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kQtThreads - 1) {
        pa[n] = ra;
        pb[n] = rb;
    }
}

struct QtNodes {  // depth l, node k at index l * n + k
    int32_t* start;
    int32_t* end;
    float2* com;
    int32_t* child;
    int32_t* nch;
};

__device__ __forceinline__ float2 centre(int32_t s, int32_t e, const float2* __restrict__ ys,
                                         const long long* __restrict__ px, const long long* __restrict__ py,
                                         const QtScal* __restrict__ sc)
{
    if (e - s == 1) return ys[s];
    const double cnt = (double)(e - s);
    const double cx = (double)sc->lo[0] + ((double)(px[e] - px[s]) / cnt) * sc->step;
    const double cy = (double)sc->lo[1] + ((double)(py[e] - py[s]) / cnt) * sc->step;
    return make_float2((float)cx, (float)cy);
}

__global__ void k_qt_root(int32_t n, QtNodes nd, const float2* __restrict__ ys, const long long* __restrict__ px,
                          const long long* __restrict__ py, QtScal* sc)
{
    nd.start[0] = 0;
    nd.end[0] = n;
    nd.com[0] = centre(0, n, ys, px, py, sc);
    nd.child[0] = -1;
    nd.nch[0] = 0;
    sc->nn[0] = 1;
}

// Depth l: a node starts at p if p is active (its depth-(l-1) node has more
// than one point) and the code prefix of 2l bits changes at p.
__global__ void k_qt_flags(const uint32_t* __restrict__ scode, const uint8_t* __restrict__ active, int32_t n,
                           int l, uint32_t* __restrict__ flag)
{
    const int shift = 32 - 2 * l;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f = 0;
        if (active[p]) {
            f = p == 0 || !active[p - 1] || (scode[p - 1] >> shift) != (scode[p] >> shift);
        }
        flag[p] = f;
    }
}

// Node ranges at depth l from the flags and their exclusive scan.
__global__ void k_qt_ranges(const uint32_t* __restrict__ scode, const uint8_t* __restrict__ active,
                            const uint32_t* __restrict__ flag, const uint32_t* __restrict__ ids, int32_t n, int l,
                            QtNodes nd, QtScal* sc)
{
    const int shift = 32 - 2 * l;
    const size_t off = (size_t)l * n;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        if (!active[p]) continue;
        const uint32_t id = ids[p] + flag[p] - 1;  // node of p
        if (flag[p]) nd.start[off + id] = (int32_t)p;
        const bool last = p == n - 1 || !active[p + 1] || (scode[p + 1] >> shift) != (scode[p] >> shift);
        if (last) nd.end[off + id] = (int32_t)p + 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->nn[l] = (int32_t)(ids[n - 1] + flag[n - 1]);
}

__global__ void k_qt_centres(int32_t n, int l, QtNodes nd, const float2* __restrict__ ys,
                             const long long* __restrict__ px, const long long* __restrict__ py,
                             const QtScal* __restrict__ sc)
{
    const int32_t nn = sc->nn[l];
    const size_t off = (size_t)l * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += (int64_t)gridDim.x * blockDim.x) {
        nd.com[off + k] = centre(nd.start[off + k], nd.end[off + k], ys, px, py, sc);
        nd.child[off + k] = -1;
        nd.nch[off + k] = 0;
    }
}

// Child links of the depth-(l-1) nodes with more than one point, and the
// active flags for depth l + 1.
__global__ void k_qt_links(const uint8_t* __restrict__ active_prev, const uint32_t* __restrict__ flag,
                           const uint32_t* __restrict__ ids, int32_t n, int l, QtNodes nd, const QtScal* __restrict__ sc,
                           uint8_t* __restrict__ active_next)
{
    const int32_t np = sc->nn[l - 1];
    const size_t po = (size_t)(l - 1) * n, co = (size_t)l * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = nd.start[po + k], e = nd.end[po + k];
        if (e - s > 1) {
            const int32_t first = (int32_t)ids[s];  // p = s starts a depth-l node
            const int32_t last = (int32_t)(ids[e - 1] + flag[e - 1]) - 1;
            nd.child[po + k] = first;
            nd.nch[po + k] = last - first + 1;
        }
    }
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        uint8_t a = 0;
        if (active_prev[p]) {
            const uint32_t id = ids[p] + flag[p] - 1;
            a = nd.end[co + id] - nd.start[co + id] > 1;
        }
        active_next[p] = a;
    }
}

// The search, one thread per point in code order.
__global__ void __launch_bounds__(kQtThreads) k_qt_search(const int32_t* __restrict__ sid,
                                                          const float2* __restrict__ ys, int32_t n, QtNodes nd,
                                                          const QtScal* __restrict__ sc, float theta, float eps,
                                                          float* __restrict__ Zp, float2* __restrict__ R,
                                                          float2* __restrict__ E, StatusBlock* st)
{
    const float ext = sc->ext;
    const float th2 = __fmul_rn(theta, theta);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float2 xi = ys[t];
        float z = 0.0f, rx = 0.0f, ry = 0.0f, ex = 0.0f, ey = 0.0f;
        auto add = [&](float2 c, float cnt) {
            const float dx = xi.x - c.x, dy = xi.y - c.y;
            const float d2 = dx * dx + dy * dy;
            const float q = 1.0f / (1.0f + d2);
            const float ke = cnt / (eps + d2);
            z += cnt * q;
            const float q2 = cnt * q * q;
            rx += q2 * dx;
            ry += q2 * dy;
            ex += ke * dx;
            ey += ke * dy;
        };
        int2 stack[kQtStack];
        int sp = 0;
        stack[sp++] = make_int2(0, 0);
        while (sp > 0) {
            const int2 top = stack[--sp];
            const int l = top.x;
            const size_t at = (size_t)l * n + top.y;
            const int32_t s = nd.start[at], e = nd.end[at];
            const bool inside = s <= t && t < e;
            if (inside && e - s == 1) continue;
            if (!inside) {
                if (e - s == 1) {
                    add(ys[s], 1.0f);
                    continue;
                }
                const float2 c = nd.com[at];
                const float w = __fmul_rn(ext, __int_as_float((127 - l) << 23));  // e 2^-l
                if (__fmul_rn(w, w) < __fmul_rn(th2, sq_rn(xi, c))) {
                    add(c, (float)(e - s));
                    continue;
                }
            }
            if (l == kQtLevels) {
                for (int32_t p = s; p < e; ++p)
                    if (p != t) add(ys[p], 1.0f);
                continue;
            }
            const int32_t first = nd.child[at], m = nd.nch[at];
            if (sp + m > kQtStack) {  // cannot happen: depth 16, at most 4 children
                record_error(st, LTSNET_ERR_DEVICE_TIMEOUT, (int32_t)t);
                break;
            }
            for (int c = m - 1; c >= 0; --c) stack[sp++] = make_int2(l + 1, first + c);
        }
        const int32_t i = sid[t];
        Zp[i] = z;
        R[i] = make_float2(rx, ry);
        E[i] = make_float2(ex, ey);
    }
}

// Exact sparse attraction A_i = sum_j p_ij (X_i - X_j) / (1 + d^2), a warp
// per row, and S = sum P_val.
__global__ void __launch_bounds__(kQtThreads) k_qt_attract(const int64_t* __restrict__ P_row,
                                                           const int32_t* __restrict__ P_col,
                                                           const float* __restrict__ P_val, int32_t n,
                                                           const float2* __restrict__ Y, float2* __restrict__ A,
                                                           StatusBlock* st)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const float2 xi = Y[i];
        float ax = 0.0f, ay = 0.0f;
        for (int64_t e = P_row[i] + lane; e < P_row[i + 1]; e += 32) {
            const int32_t j = P_col[e];
            if ((uint32_t)j >= (uint32_t)n) {
                record_error(st, LTSNET_ERR_BAD_GRAPH, j);
                continue;
            }
            const float2 xj = Y[j];
            const float dx = xi.x - xj.x, dy = xi.y - xj.y;
            const float k = P_val[e] / (1.0f + dx * dx + dy * dy);
            ax += k * dx;
            ay += k * dy;
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if (lane == 0) A[i] = make_float2(ax, ay);
    }
}

// Fixed-order FP64 sums of Zp and P_val: per-block partials.
__global__ void __launch_bounds__(kQtThreads) k_qt_partials(const float* __restrict__ Zp, int32_t n,
                                                            const float* __restrict__ P_val, int64_t nnz,
                                                            double* __restrict__ part)
{
    double z = 0.0, s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z += (double)Zp[i];
    if (P_val)
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
            s += (double)P_val[e];
    z = warp_sum(z);
    s = warp_sum(s);
    __shared__ double rz[kQtThreads / 32], rs[kQtThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        rz[threadIdx.x >> 5] = z;
        rs[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kQtThreads / 32; ++q) {
            z += rz[q];
            s += rs[q];
        }
        part[2 * blockIdx.x] = z;
        part[2 * blockIdx.x + 1] = s;
    }
}

// Z and S: BH variant from the partials; FIt variant Z, S from the grid
// gradient's terms (f64: Z, S, ...).
__global__ void k_qt_scalars(const double* __restrict__ part, int32_t nparts, const double* __restrict__ grid_terms,
                             double* __restrict__ zs)
{
    if (grid_terms) {
        zs[0] = grid_terms[0];
        zs[1] = grid_terms[1];
        return;
    }
    double z = 0.0, s = 0.0;
    for (int q = 0; q < nparts; ++q) {
        z += part[2 * q];
        s += part[2 * q + 1];
    }
    zs[0] = z;
    zs[1] = s;
}

struct QtCoef {
    float a_att, a_rep, a_cmp, a_ent;
};

// g = a_att A - a_rep (S/Z) R + a_cmp X - a_ent E; A and R from `parts`
// (f32 [n][6]: A, R, E) when given, else from A / R.
__global__ void k_qt_assemble(const float2* __restrict__ Y, int32_t n, const float2* __restrict__ A,
                              const float2* __restrict__ R, const float* __restrict__ grid_parts,
                              const float2* __restrict__ E, const double* __restrict__ zs, QtCoef c,
                              float2* __restrict__ grad, float* __restrict__ parts_out)
{
    const float soz = (float)(zs[1] / zs[0]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 a, r;
        if (grid_parts) {
            a = make_float2(grid_parts[6 * i], grid_parts[6 * i + 1]);
            r = make_float2(grid_parts[6 * i + 2], grid_parts[6 * i + 3]);
        } else {
            a = A[i];
            r = R[i];
        }
        const float2 e = E[i], y = Y[i];
        grad[i] = make_float2(c.a_att * a.x - c.a_rep * soz * r.x + c.a_cmp * y.x - c.a_ent * e.x,
                              c.a_att * a.y - c.a_rep * soz * r.y + c.a_cmp * y.y - c.a_ent * e.y);
        if (parts_out) {
            parts_out[6 * i] = a.x;
            parts_out[6 * i + 1] = a.y;
            parts_out[6 * i + 2] = r.x;
            parts_out[6 * i + 3] = r.y;
            parts_out[6 * i + 4] = e.x;
            parts_out[6 * i + 5] = e.y;
        }
    }
}

// The descent step of every variant (the same rule as ltsnet_optimize): a
// gain grows by 0.2 where the gradient's sign differs from the previous
// step's, else shrinks by x0.8, floored at 0.01; step = momentum step -
// lr gain grad; Y += step.
__device__ __forceinline__ float sign_of(float x) { return (float)((x > 0.0f) - (x < 0.0f)); }

__global__ void k_qt_step(int32_t n, float2* __restrict__ Y, float2* __restrict__ upd, float2* __restrict__ gains,
                          const float2* __restrict__ grad, float momentum, float lr, StatusBlock* st)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 g = grad[i];
        float2 u = upd[i], gn = gains[i], y = Y[i];
        gn.x = sign_of(g.x) != sign_of(u.x) ? gn.x + 0.2f : gn.x * 0.8f;
        gn.y = sign_of(g.y) != sign_of(u.y) ? gn.y + 0.2f : gn.y * 0.8f;
        gn.x = fmaxf(gn.x, 0.01f);
        gn.y = fmaxf(gn.y, 0.01f);
        u.x = momentum * u.x - lr * gn.x * g.x;
        u.y = momentum * u.y - lr * gn.y * g.y;
        y.x += u.x;
        y.y += u.y;
        if (!(isfinite(y.x) && isfinite(y.y))) record_error(st, LTSNET_ERR_NONFINITE, (int32_t)i);
        upd[i] = u;
        gains[i] = gn;
        Y[i] = y;
    }
}

struct QtWs {
    StatusBlock* st;
    QtScal* sc;
    uint64_t *k0, *k1;
    double *v0, *v1;
    uint32_t* hist;
    uint32_t* tmp;
    int32_t* sid;
    float2* ys;
    uint32_t* scode;
    long long *qx, *qy, *px, *py;
    long long* bs;
    uint8_t *act0, *act1;
    uint32_t *flag, *ids;
    QtNodes nd;
    float* Zp;
    float2 *R, *E, *A;
    double* part;
    double* zs;
    float* gparts;   // FIt: the grid gradient's parts (f32 [n][6])
    double* gterms;  // FIt: its terms (f64 [8])
    float* ggrad;    // FIt: its gradient (unused)
    void* gws;       // FIt: its workspace
    size_t gws_bytes;
};

size_t qt_carve(void* ws, int32_t n, size_t grid_ws, QtWs* w)
{
    Carve c(ws, ~(size_t)0);
    QtWs t;
    const size_t L = kQtLevels + 1;
    t.st = c.take<StatusBlock>(1);
    t.sc = c.take<QtScal>(1);
    t.k0 = c.take<uint64_t>(n);
    t.k1 = c.take<uint64_t>(n);
    t.v0 = c.take<double>(n);
    t.v1 = c.take<double>(n);
    t.hist = c.take<uint32_t>(radix_hist_words(n));
    t.tmp = c.take<uint32_t>(std::max(scan_tmp_words(radix_hist_words(n)), scan_tmp_words(n)));
    t.sid = c.take<int32_t>(n);
    t.ys = c.take<float2>(n);
    t.scode = c.take<uint32_t>(n);
    t.qx = c.take<long long>(n);
    t.qy = c.take<long long>(n);
    t.px = c.take<long long>((size_t)n + 1);
    t.py = c.take<long long>((size_t)n + 1);
    t.bs = c.take<long long>(2 * ((size_t)n / kScanChunk + 1));
    t.act0 = c.take<uint8_t>(n);
    t.act1 = c.take<uint8_t>(n);
    t.flag = c.take<uint32_t>(n);
    t.ids = c.take<uint32_t>(n);
    t.nd.start = c.take<int32_t>(L * n);
    t.nd.end = c.take<int32_t>(L * n);
    t.nd.com = c.take<float2>(L * n);
    t.nd.child = c.take<int32_t>(L * n);
    t.nd.nch = c.take<int32_t>(L * n);
    t.Zp = c.take<float>(n);
    t.R = c.take<float2>(n);
    t.E = c.take<float2>(n);
    t.A = c.take<float2>(n);
    t.part = c.take<double>(2 * kQtBlocks);
    t.zs = c.take<double>(2);
    t.gparts = grid_ws ? c.take<float>((size_t)6 * n) : nullptr;
    t.gterms = grid_ws ? c.take<double>(8) : nullptr;
    t.ggrad = grid_ws ? c.take<float>((size_t)2 * n) : nullptr;
    t.gws = grid_ws ? c.take<unsigned char>(grid_ws) : nullptr;
    t.gws_bytes = grid_ws;
    if (w) *w = t;
    return align_up(c.off, 256);
}

// Builds the tree of Y and runs the search: Zp, R, E per point.
ltsnet_status qt_sums(const float2* Y, int32_t n, float theta, float eps, const QtWs& w, cudaStream_t s)
{
    const unsigned fb = kQtBlocks;
    QtScal init{};
    init.lo_ord[0] = init.lo_ord[1] = 0x7fffffff;
    init.hi_ord[0] = init.hi_ord[1] = (int32_t)0x80000000;
    LT_CUDA(cudaMemcpyAsync(w.sc, &init, sizeof(QtScal), cudaMemcpyHostToDevice, s));
    k_qt_bounds<<<fb, kQtThreads, 0, s>>>(Y, n, w.sc);
    k_qt_domain<<<1, 1, 0, s>>>(w.sc);
    k_qt_codes<<<fb, kQtThreads, 0, s>>>(Y, n, w.sc, w.k0);
    count_launches(3);
    LT_CHECK_LAUNCH();
    bool alt = false;
    LT_CUDA(radix_sort_u64_f64(w.k0, w.v0, w.k1, w.v1, n, 32, w.hist, w.tmp, s, &alt));
    k_qt_gather<<<fb, kQtThreads, 0, s>>>(alt ? w.k1 : w.k0, Y, n, w.sc, w.sid, w.ys, w.scode, w.qx, w.qy, w.act0);
    const int nb = (int)(((int64_t)n + kScanChunk - 1) / kScanChunk);
    k_scan64_reduce<<<nb, kQtThreads, 0, s>>>(w.qx, w.qy, n, w.bs);
    k_scan64_top<<<1, 1, 0, s>>>(w.bs, nb);
    k_scan64_down<<<nb, kQtThreads, 0, s>>>(w.qx, w.qy, n, w.bs, w.px, w.py);
    k_qt_root<<<1, 1, 0, s>>>(n, w.nd, w.ys, w.px, w.py, w.sc);
    count_launches(5);
    LT_CHECK_LAUNCH();
    uint8_t* act = w.act0;
    uint8_t* nxt = w.act1;
    for (int l = 1; l <= kQtLevels; ++l) {
        k_qt_flags<<<fb, kQtThreads, 0, s>>>(w.scode, act, n, l, w.flag);
        count_launches(1);
        LT_CUDA(scan_u32_exclusive(w.flag, w.ids, n, w.tmp, s));
        k_qt_ranges<<<fb, kQtThreads, 0, s>>>(w.scode, act, w.flag, w.ids, n, l, w.nd, w.sc);
        k_qt_centres<<<fb, kQtThreads, 0, s>>>(n, l, w.nd, w.ys, w.px, w.py, w.sc);
        k_qt_links<<<fb, kQtThreads, 0, s>>>(act, w.flag, w.ids, n, l, w.nd, w.sc, nxt);
        count_launches(3);
        LT_CHECK_LAUNCH();
        std::swap(act, nxt);
    }
    k_qt_search<<<(unsigned)((n + kQtThreads - 1) / kQtThreads), kQtThreads, 0, s>>>(w.sid, w.ys, n, w.nd, w.sc, theta,
                                                                                      eps, w.Zp, w.R, w.E, w.st);
    count_launches(1);
    LT_CHECK_LAUNCH();
    return LTSNET_OK;
}

}  // namespace
}  // namespace lt

extern "C" size_t ltsnet_gradient_quadtree_workspace_size(int32_t n, const ltsnet_params* p, int32_t variant)
{
    if (n < 1 || (variant != LTSNET_VARIANT_BH && variant != LTSNET_VARIANT_FIT)) return 0;
    size_t g = 0;
    if (variant == LTSNET_VARIANT_FIT) {
        if (!p) return 0;
        g = ltsnet_gradient_workspace_size(n, p);
        if (g == 0) return 0;
    }
    return lt::qt_carve(nullptr, n, g, nullptr);
}

extern "C" ltsnet_status ltsnet_gradient_quadtree(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                                                  int32_t n, const float* Y, const ltsnet_stage* stage,
                                                  const ltsnet_params* p, float theta, int32_t variant, float* grad,
                                                  float* parts, double* terms, void* ws, size_t ws_bytes,
                                                  ltsnet_stream stream)
{
    using namespace lt;
    if (n < 2 || !P_row || !P_col || !P_val || !Y || !stage || !p || !grad || !ws || !(theta >= 0.0f) ||
        !isfinite(theta) || (variant != LTSNET_VARIANT_BH && variant != LTSNET_VARIANT_FIT))
        return LTSNET_ERR_INVALID_ARG;
    const size_t need = ltsnet_gradient_quadtree_workspace_size(n, p, variant);
    if (need == 0) return LTSNET_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255) || ws_bytes < need) return LTSNET_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t g = variant == LTSNET_VARIANT_FIT ? ltsnet_gradient_workspace_size(n, p) : 0;
    QtWs w;
    qt_carve(ws, n, g, &w);
    const float2* Y2 = (const float2*)Y;
    LT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StatusBlock), s));
    if (variant == LTSNET_VARIANT_FIT) {
        // A, R, Z and S from the grid interpolation (its E is not used)
        ltsnet_status e = ltsnet_gradient(P_row, P_col, P_val, n, Y, stage, p, w.ggrad, w.gparts, w.gterms, w.gws,
                                          w.gws_bytes, stream);
        if (e != LTSNET_OK) return e;
        ltsnet_status ge = ltsnet_poll_status(w.gws, w.gws_bytes, stream);
        if (ge < 0) return ge;
    }
    if (ltsnet_status e = qt_sums(Y2, n, theta, p->eps, w, s)) return e;
    int64_t nnz_host = 0;
    if (variant == LTSNET_VARIANT_BH) {
        k_qt_attract<<<kQtBlocks, kQtThreads, 0, s>>>(P_row, P_col, P_val, n, Y2, w.A, w.st);
        count_launches(1);
        LT_CHECK_LAUNCH();
        LT_CUDA(cudaMemcpyAsync(&nnz_host, P_row + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LT_CUDA(cudaStreamSynchronize(s));
    }
    k_qt_partials<<<kQtBlocks, kQtThreads, 0, s>>>(w.Zp, n, variant == LTSNET_VARIANT_BH ? P_val : nullptr, nnz_host,
                                                   w.part);
    k_qt_scalars<<<1, 1, 0, s>>>(w.part, kQtBlocks, variant == LTSNET_VARIANT_FIT ? w.gterms : nullptr, w.zs);
    QtCoef c;
    c.a_att = (float)(4.0 * (double)stage->lambda_kl * (double)stage->exaggeration);
    c.a_rep = (float)(4.0 * (double)stage->lambda_kl);
    c.a_cmp = (float)((double)stage->lambda_c / (double)n);
    c.a_ent = (float)((double)stage->lambda_r / ((double)n * (double)n));
    k_qt_assemble<<<kQtBlocks, kQtThreads, 0, s>>>(Y2, n, w.A, w.R, variant == LTSNET_VARIANT_FIT ? w.gparts : nullptr,
                                                   w.E, w.zs, c, (float2*)grad, parts);
    count_launches(3);
    LT_CHECK_LAUNCH();
    StatusBlock hs;
    double zs[2];
    LT_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaMemcpyAsync(zs, w.zs, sizeof(zs), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    if (terms) {
        terms[0] = zs[0];
        terms[1] = zs[1];
    }
    if (hs.code) return (ltsnet_status)hs.code;
    return LTSNET_OK;
}

extern "C" size_t ltsnet_optimize_quadtree_workspace_size(int32_t n, const ltsnet_params* p, int32_t variant)
{
    const size_t g = ltsnet_gradient_quadtree_workspace_size(n, p, variant);
    if (g == 0) return 0;
    return lt::align_up(sizeof(lt::StatusBlock) + sizeof(float) * 2 * (size_t)n, 256) + g;
}

extern "C" ltsnet_status ltsnet_optimize_quadtree(const int64_t* P_row, const int32_t* P_col, const float* P_val,
                                                  int32_t n, const ltsnet_params* p, float theta, int32_t variant,
                                                  float* Y, float* update, float* gains, int32_t start_iter,
                                                  int32_t n_iter, void* ws, size_t ws_bytes, ltsnet_stream stream)
{
    using namespace lt;
    if (!p || p->n_stages < 1 || !p->stages || !Y || !update || !gains || start_iter < 0 || n_iter < 0)
        return LTSNET_ERR_INVALID_ARG;
    const size_t need = ltsnet_optimize_quadtree_workspace_size(n, p, variant);
    if (need == 0) return LTSNET_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255) || ws_bytes < need) return LTSNET_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Carve c(ws, ws_bytes);
    StatusBlock* st = c.take<StatusBlock>(1);
    float* grad = c.take<float>((size_t)2 * n);
    const size_t gofs = align_up(c.off, 256);
    void* gws = (char*)ws + gofs;
    const size_t gbytes = ws_bytes - gofs;
    LT_CUDA(cudaMemsetAsync(st, 0, sizeof(StatusBlock), s));
    const float lr = p->learning_rate > 0.f ? p->learning_rate : std::max(200.0f, (float)n / 12.0f);
    for (int64_t t = start_iter; t < (int64_t)start_iter + n_iter; ++t) {
        // the stage of iteration t; past the schedule's end, the last stage
        const ltsnet_stage* sg = &p->stages[p->n_stages - 1];
        int64_t acc = 0;
        for (int q = 0; q < p->n_stages; ++q) {
            acc += p->stages[q].iters;
            if (t < acc) {
                sg = &p->stages[q];
                break;
            }
        }
        ltsnet_status e = ltsnet_gradient_quadtree(P_row, P_col, P_val, n, Y, sg, p, theta, variant, grad, nullptr,
                                                   nullptr, gws, gbytes, stream);
        if (e < 0) return e;
        k_qt_step<<<kQtBlocks, kQtThreads, 0, s>>>(n, (float2*)Y, (float2*)update, (float2*)gains,
                                                   (const float2*)grad, sg->momentum, lr, st);
        count_launches(1);
        LT_CHECK_LAUNCH();
    }
    StatusBlock hs;
    LT_CUDA(cudaMemcpyAsync(&hs, st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    return hs.code ? (ltsnet_status)hs.code : LTSNET_OK;
}
