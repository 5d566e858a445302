// Layout quality metrics of Sec. 4 ("Quality Metrics Comparison"):
// neighbourhood preservation with r = 2 and stress.
//
// NP: for every vertex v, b = |N_G(v, 2)| (vertices within two hops, v
// excluded) and c = |N_G(v, 2) cap N_D(v)|, N_D(v) being the b vertices
// nearest to v in the drawing; NP is the mean of c / (2b - c) over the
// vertices with b > 0.  "Nearest" orders the keys
// (FP32 squared distance, vertex id): dx = x_u - x_v, dy = y_u - y_v,
// dx*dx + dy*dy with every operation rounded on its own, ties to the smaller
// id.  Every vertex counts, hubs of scale-free graphs included.
//
// Per vertex, one warp: (1) the 2-hop ball goes into a hash set -- in shared
// memory (4096 slots) when its candidate count deg(v) + sum of deg(w) over
// the adjacency entries w is at most 2048, else in a table of at least twice
// the candidate count (a power of two) in a global pool, those vertices
// being listed by the first pass and processed in batches that fit the
// pool; (2) a uniform grid of square cells over the drawing, its points
// sorted by cell and a summed-area table of the cell counts, gives the
// smallest square of cells around v holding b other points; every point
// within sqrt(2) times that square's reach lies in a wider square of
// cells, so the b nearest are among its points; (3) a radix select over
// the 64-bit keys of those candidates finds the b-th smallest key T; (4) c
// counts the candidates with key <= T that are in the hash set.
//
// Stress: for every source s, a BFS (bfs_levels.cuh) and one pass over the
// vertices accumulate r = ||X_s - X_j|| / d_sj, r^2 and the pair counts in
// FP64; each block keeps its own running sums across sources and one block
// adds them in a fixed order, so the result is reproducible.  The host
// returns ST = 1 - (sum r)^2 / (N sum r^2) at the optimal scale
// alpha = sum r / sum r^2.
#include <math.h>

#include <algorithm>
#include <vector>

#include "bfs_levels.cuh"

namespace lt {
namespace {

constexpr int kQThreads = 256;
constexpr int kNpWarps = 2;          // warps per block of the NP kernel
constexpr int kNpCap = 2048;         // 2-hop candidates (with repeats) of a shared-memory ball
constexpr int kHashSlots = 4096;     // >= 2 kNpCap: load factor <= 1/2
constexpr int kHashBits = 12;
constexpr int kQBlocks = kSplitBlocks * 4;  // fixed: sizes workspace and host partials

struct QualityScal {
    int32_t lo_ord[2];  // f2ord of the drawing's min x, min y
    int32_t hi_ord[2];  // f2ord of max x, max y
    int32_t G;          // cells per side
    float lo[2], h, inv_h;
    int32_t nlarge;     // vertices whose ball goes to the global pool
    int32_t pad[6];
};

struct StressAcc {
    double s1, s2;
    unsigned long long cnt, skipped;
};

__device__ __forceinline__ float sq_dist_rn(float2 a, float2 b)
{
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// ---------------------------------------------------------------------------
// Uniform grid over the drawing.

__global__ void k_q_bounds(const float2* __restrict__ Y, int32_t n, QualityScal* sc)
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

__global__ void k_q_grid(QualityScal* sc, int32_t n, int32_t G)
{
    const float lx = ord2f(sc->lo_ord[0]), ly = ord2f(sc->lo_ord[1]);
    const float ext = fmaxf(fmaxf(ord2f(sc->hi_ord[0]) - lx, ord2f(sc->hi_ord[1]) - ly), 1e-30f);
    sc->G = G;
    sc->lo[0] = lx;
    sc->lo[1] = ly;
    sc->h = ext / (float)G;
    sc->inv_h = (float)G / ext;
    sc->nlarge = 0;
}

__device__ __forceinline__ int cell_of(float v, float lo, float inv_h, int G)
{
    const int c = (int)((v - lo) * inv_h);
    return min(max(c, 0), G - 1);
}

__global__ void k_q_count(const float2* __restrict__ Y, int32_t n, const QualityScal* __restrict__ sc,
                          int32_t* __restrict__ cnt, int32_t* __restrict__ cell)
{
    const int G = sc->G;
    const float lx = sc->lo[0], ly = sc->lo[1], ih = sc->inv_h;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 y = Y[i];
        const int c = cell_of(y.y, ly, ih, G) * G + cell_of(y.x, lx, ih, G);
        cell[i] = c;
        atomicAdd(&cnt[c], 1);
    }
}

// Exclusive scan of the cell counts into start[0..G*G] (one block).
__global__ void __launch_bounds__(1024) k_q_scan(const int32_t* __restrict__ cnt, int32_t ncell,
                                                 int32_t* __restrict__ start, int32_t* __restrict__ cursor)
{
    __shared__ int32_t part[1024];
    const int per = (ncell + 1023) / 1024;
    const int a = threadIdx.x * per, b = min(ncell, a + per);
    int32_t s = 0;
    for (int i = a; i < b; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int t = 0; t < 1024; ++t) {
            const int32_t v = part[t];
            part[t] = run;
            run += v;
        }
        start[ncell] = run;
    }
    __syncthreads();
    s = part[threadIdx.x];
    for (int i = a; i < b; ++i) {
        start[i] = s;
        cursor[i] = s;
        s += cnt[i];
    }
}

__global__ void k_q_scatter(const float2* __restrict__ Y, int32_t n, const int32_t* __restrict__ cell,
                            int32_t* __restrict__ cursor, int32_t* __restrict__ sid, float2* __restrict__ sy)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pos = atomicAdd(&cursor[cell[i]], 1);
        sid[pos] = (int32_t)i;
        sy[pos] = Y[i];
    }
}

// Summed-area table: sat[y][x] = counts over cells [0..y] x [0..x].
__global__ void k_q_sat_rows(const int32_t* __restrict__ cnt, int32_t G, int32_t* __restrict__ sat)
{
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < G; y += gridDim.x * blockDim.x) {
        int32_t s = 0;
        for (int x = 0; x < G; ++x) {
            s += cnt[(size_t)y * G + x];
            sat[(size_t)y * G + x] = s;
        }
    }
}

__global__ void k_q_sat_cols(int32_t G, int32_t* __restrict__ sat)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < G; x += gridDim.x * blockDim.x) {
        int32_t s = 0;
        for (int y = 0; y < G; ++y) {
            s += sat[(size_t)y * G + x];
            sat[(size_t)y * G + x] = s;
        }
    }
}

__device__ __forceinline__ int32_t sat_box(const int32_t* __restrict__ sat, int G, int x0, int x1, int y0, int y1)
{
    auto at = [&](int y, int x) -> int32_t { return (x < 0 || y < 0) ? 0 : sat[(size_t)y * G + x]; };
    return at(y1, x1) - at(y0 - 1, x1) - at(y1, x0 - 1) + at(y0 - 1, x0 - 1);
}

// ---------------------------------------------------------------------------
// NP, one warp per vertex.

__device__ __forceinline__ uint32_t hash_slot(int32_t u, int bits)
{
    return ((uint32_t)u * 2654435761u) >> (32 - bits);
}

// Inserts u into the table of 2^bits slots (shared or global memory);
// returns 1 if it was not there.  The load factor is at most 1/2.
__device__ __forceinline__ int hash_insert(int32_t* h, int bits, int32_t u)
{
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hash_slot(u, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t old = atomicCAS(&h[s], -1, u);
        if (old == -1) return 1;
        if (old == u) return 0;
        s = (s + 1) & mask;
    }
    return 0;  // unreachable at load factor <= 1/2
}

__device__ __forceinline__ bool hash_has(const int32_t* h, int bits, int32_t u)
{
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hash_slot(u, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t x = ((const volatile int32_t*)h)[s];
        if (x == u) return true;
        if (x == -1) return false;
        s = (s + 1) & mask;
    }
    return false;
}

__device__ __forceinline__ unsigned long long np_key(float2 p, float2 v, int32_t u)
{
    return ((unsigned long long)__float_as_uint(sq_dist_rn(p, v)) << 32) | (uint32_t)u;
}

struct NpArgs {
    const int64_t* row_ptr;
    const int32_t* col;
    int32_t n;
    const float2* Y;
    const QualityScal* sc;
    const int32_t* start;
    const int32_t* sat;
    const int32_t* sid;
    const float2* sy;
    int32_t* ball;
    int32_t* common;
    StatusBlock* st;
};

// Steps (1)-(4) for vertex v by one warp, with the 2-hop ball in the empty
// table h of 2^bits slots (cleared again before returning) and a 256-bin
// histogram hg in shared memory.
__device__ void np_vertex(const NpArgs& A, int64_t v, int32_t* h, int bits, uint32_t* hg, int lane)
{
    const int64_t* __restrict__ row_ptr = A.row_ptr;
    const int32_t* __restrict__ col = A.col;
    const int32_t n = A.n;
    const int64_t a0 = row_ptr[v], a1 = row_ptr[v + 1];
    int added = 0;
    for (int64_t e = a0 + lane; e < a1; e += 32) {
        const int32_t x = col[e];
        if ((uint32_t)x >= (uint32_t)n) {
            record_error(A.st, LTSNET_ERR_BAD_GRAPH, x);
            continue;
        }
        if (x != v) added += hash_insert(h, bits, x);
    }
    for (int64_t e = a0; e < a1; ++e) {
        const int32_t x = col[e];
        if ((uint32_t)x >= (uint32_t)n) continue;
        const int64_t b0 = row_ptr[x], b1 = row_ptr[x + 1];
        for (int64_t f = b0 + lane; f < b1; f += 32) {
            const int32_t u = col[f];
            if ((uint32_t)u >= (uint32_t)n) {
                record_error(A.st, LTSNET_ERR_BAD_GRAPH, u);
                continue;
            }
            if (u != v) added += hash_insert(h, bits, u);
        }
    }
    __syncwarp();
    int32_t b = added;
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(FULL, b, o);
    int32_t c = 0;
    if (b > 0) {
        const QualityScal* sc = A.sc;
        const int G = sc->G;
        const float lx = sc->lo[0], ly = sc->lo[1], ih = sc->inv_h;
        const int32_t* __restrict__ start = A.start;
        const int32_t* __restrict__ sid = A.sid;
        const float2* __restrict__ sy = A.sy;
        // (2) the smallest square of cells around v with b other points
        const float2 yv = A.Y[v];
        const int cx = cell_of(yv.x, lx, ih, G), cy = cell_of(yv.y, ly, ih, G);
        // at R = G - 1 the square is the whole grid (n >= b + 1 points), so
        // the cap never binds; it keeps the loop bounded by construction
        int R = 0;
        while (R < G - 1 &&
               sat_box(A.sat, G, max(cx - R, 0), min(cx + R, G - 1), max(cy - R, 0), min(cy + R, G - 1)) < b + 1)
            ++R;
        // every point of that square lies within sqrt(2) (R + 1) cell
        // widths of v, or (R + 2) where rounding put a point or v one cell
        // off; one cell more on the way back out for the same reason
        const int Rw = (int)ceilf(1.41421357f * (float)(R + 2)) + 1;
        const int x0 = max(cx - Rw, 0), x1 = min(cx + Rw, G - 1);
        const int y0 = max(cy - Rw, 0), y1 = min(cy + Rw, G - 1);
        // (3) radix select of the b-th smallest key among the candidates
        unsigned long long prefix = 0;
        uint32_t rank = (uint32_t)b;  // 1-based
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int i = lane; i < 256; i += 32) hg[i] = 0;
            __syncwarp();
            const unsigned long long himask = shift == 56 ? 0ull : (~0ull << (shift + 8));
            for (int yy = y0; yy <= y1; ++yy) {
                const int32_t p0 = start[(size_t)yy * G + x0], p1 = start[(size_t)yy * G + x1 + 1];
                for (int32_t p = p0 + lane; p < p1; p += 32) {
                    const int32_t u = sid[p];
                    if (u == v) continue;
                    const unsigned long long key = np_key(sy[p], yv, u);
                    if ((key & himask) == prefix) atomicAdd(&hg[(key >> shift) & 255], 1u);
                }
            }
            __syncwarp();
            // bin holding the rank-th key (every lane scans the same 256 bins)
            uint32_t run = 0;
            int bin = 255;
            for (int q = 0; q < 256; ++q) {
                const uint32_t cq = hg[q];
                if (run + cq >= rank) {
                    bin = q;
                    break;
                }
                run += cq;
            }
            rank -= run;
            prefix |= (unsigned long long)bin << shift;
            __syncwarp();
        }
        // (4) candidates with key <= T that are in the ball
        for (int yy = y0; yy <= y1; ++yy) {
            const int32_t p0 = start[(size_t)yy * G + x0], p1 = start[(size_t)yy * G + x1 + 1];
            for (int32_t p = p0 + lane; p < p1; p += 32) {
                const int32_t u = sid[p];
                if (u == v) continue;
                if (np_key(sy[p], yv, u) <= prefix && hash_has(h, bits, u)) ++c;
            }
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    }
    if (lane == 0) {
        A.ball[v] = b;
        A.common[v] = c;
    }
    __syncwarp();
    for (int64_t i = lane; i < ((int64_t)1 << bits); i += 32) h[i] = -1;
    __syncwarp();
}

// Every vertex: candidate count; balls of at most kNpCap candidates in a
// shared-memory table, the others listed (vertex, candidates) for
// k_np_large.
__global__ void __launch_bounds__(kNpWarps * 32) k_np(NpArgs A, QualityScal* sc, int32_t* __restrict__ large_v,
                                                      int64_t* __restrict__ large_cand)
{
    __shared__ int32_t hs[kNpWarps][kHashSlots];
    __shared__ uint32_t hist[kNpWarps][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t* h = hs[w];
    uint32_t* hg = hist[w];
    for (int i = lane; i < kHashSlots; i += 32) h[i] = -1;
    __syncwarp();
    const int64_t nw = (int64_t)gridDim.x * kNpWarps;
    for (int64_t v = (int64_t)blockIdx.x * kNpWarps + w; v < A.n; v += nw) {
        const int64_t a0 = A.row_ptr[v], a1 = A.row_ptr[v + 1];
        long long cand = lane == 0 ? a1 - a0 : 0;  // deg(v) once, then the neighbours' degrees
        for (int64_t e = a0 + lane; e < a1; e += 32) {
            const int32_t x = A.col[e];
            if ((uint32_t)x < (uint32_t)A.n) cand += A.row_ptr[x + 1] - A.row_ptr[x];
        }
        for (int o = 16; o > 0; o >>= 1) cand += __shfl_xor_sync(FULL, cand, o);
        if (cand > kNpCap) {
            if (lane == 0) {
                const int32_t slot = atomicAdd(&sc->nlarge, 1);
                large_v[slot] = (int32_t)v;
                large_cand[slot] = cand;
            }
            continue;
        }
        np_vertex(A, v, h, kHashBits, hg, lane);
    }
}

// The listed vertices lv[0..count), one warp each, every ball in its own
// table of 2^bits[i] slots at pool + off[i] (empty on entry: the host clears
// the pool once per call and every vertex clears its table after use).
__global__ void __launch_bounds__(kNpWarps * 32) k_np_large(NpArgs A, const int32_t* __restrict__ lv,
                                                            const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ bits, int32_t count,
                                                            int32_t* __restrict__ pool)
{
    __shared__ uint32_t hist[kNpWarps][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kNpWarps;
    for (int64_t i = (int64_t)blockIdx.x * kNpWarps + w; i < count; i += nw) {
        np_vertex(A, lv[i], pool + off[i], bits[i], hist[w], lane);
    }
}

// NP = mean over b > 0 of c / (2b - c); fixed summation order.
__global__ void __launch_bounds__(kQThreads) k_np_partial(const int32_t* __restrict__ ball,
                                                          const int32_t* __restrict__ common, int32_t n,
                                                          double* __restrict__ part, unsigned long long* __restrict__ pcnt)
{
    __shared__ double rs[kQThreads / 32];
    __shared__ unsigned long long rc[kQThreads / 32];
    double s = 0.0;
    unsigned long long k = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = ball[i];
        if (b > 0) {
            const int32_t c = common[i];
            s += (double)c / (double)(2 * b - c);
            ++k;
        }
    }
    s = warp_sum(s);
    k = warp_sum(k);
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = s;
        rc[threadIdx.x >> 5] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long kt = 0;
        for (int q = 0; q < kQThreads / 32; ++q) {
            t += rs[q];
            kt += rc[q];
        }
        part[blockIdx.x] = t;
        pcnt[blockIdx.x] = kt;
    }
}

// ---------------------------------------------------------------------------
// Stress.

__global__ void k_stress_seed(const int32_t* __restrict__ sources, int32_t s, int32_t n, uint16_t* __restrict__ D,
                              int32_t* __restrict__ q0, LevelCtl* ctl, StatusBlock* st)
{
    const int32_t src = sources[s];
    if ((uint32_t)src >= (uint32_t)n) {
        record_error(st, LTSNET_ERR_INVALID_ARG, s);
        ctl->cnt[0] = ctl->cnt[1] = 0;
        ctl->err = 3;
        return;
    }
    bfs_seed(ctl, D, n, 0, src, q0);
}

// Each block adds its share of source s's pairs to its own running sums.
__global__ void __launch_bounds__(kQThreads) k_stress_accum(const uint16_t* __restrict__ d,
                                                            const float2* __restrict__ Y, int32_t n,
                                                            const int32_t* __restrict__ sources, int32_t s,
                                                            StressAcc* __restrict__ acc)
{
    __shared__ double r1[kQThreads / 32], r2[kQThreads / 32];
    __shared__ unsigned long long rc[kQThreads / 32], rk[kQThreads / 32];
    const int32_t src = sources[s];
    const float2 ys = Y[src];
    double s1 = 0.0, s2 = 0.0;
    unsigned long long cnt = 0, skipped = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t dj = d[i];
        if (dj == kUnreached) {
            ++skipped;
        } else if (dj > 0) {
            const float2 y = Y[i];
            const double dx = (double)y.x - (double)ys.x, dy = (double)y.y - (double)ys.y;
            const double r = sqrt(dx * dx + dy * dy) / (double)dj;
            s1 += r;
            s2 += r * r;
            ++cnt;
        }
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    cnt = warp_sum(cnt);
    skipped = warp_sum(skipped);
    if ((threadIdx.x & 31) == 0) {
        const int q = threadIdx.x >> 5;
        r1[q] = s1;
        r2[q] = s2;
        rc[q] = cnt;
        rk[q] = skipped;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        StressAcc a = acc[blockIdx.x];
        for (int q = 0; q < kQThreads / 32; ++q) {
            a.s1 += r1[q];
            a.s2 += r2[q];
            a.cnt += rc[q];
            a.skipped += rk[q];
        }
        acc[blockIdx.x] = a;
    }
}

struct QualityWs {
    StatusBlock* st;
    QualityScal* sc;
    LevelCtl* ctl;
    int32_t* cnt;     // G*G
    int32_t* start;   // G*G + 1
    int32_t* cursor;  // G*G
    int32_t* sat;     // G*G
    int32_t* cell;    // n
    int32_t* sid;     // n
    float2* sy;       // n
    int32_t* ball;    // n
    int32_t* common;  // n
    uint16_t* D;      // n
    int32_t* q0;      // n
    int32_t* q1;      // n
    double* part;
    unsigned long long* pcnt;
    StressAcc* acc;
    int32_t* lv;      // n: vertices of the global-pool path
    int64_t* lcand;   // n: their candidate counts, then their table offsets
    int32_t* lbits;   // n: their table sizes (log2)
    int32_t* pool;    // the rest of the workspace: hash tables of those vertices
    int64_t pool_slots;
};

int32_t grid_side(int32_t n) { return std::max(1, (int32_t)ceil(sqrt((double)n / 2.0))); }

size_t quality_carve(void* ws, int32_t n, QualityWs* w)
{
    const int32_t G = grid_side(n);
    const size_t cells = (size_t)G * G;
    Carve c(ws, ~(size_t)0);
    QualityWs t;
    t.st = c.take<StatusBlock>(1);
    t.sc = c.take<QualityScal>(1);
    t.ctl = c.take<LevelCtl>(1);
    t.cnt = c.take<int32_t>(cells);
    t.start = c.take<int32_t>(cells + 1);
    t.cursor = c.take<int32_t>(cells);
    t.sat = c.take<int32_t>(cells);
    t.cell = c.take<int32_t>(n);
    t.sid = c.take<int32_t>(n);
    t.sy = c.take<float2>(n);
    t.ball = c.take<int32_t>(n);
    t.common = c.take<int32_t>(n);
    t.D = c.take<uint16_t>(n);
    t.q0 = c.take<int32_t>(n);
    t.q1 = c.take<int32_t>(n);
    t.part = c.take<double>(kQBlocks);
    t.pcnt = c.take<unsigned long long>(kQBlocks);
    t.acc = c.take<StressAcc>(kQBlocks);
    t.lv = c.take<int32_t>(n);
    t.lcand = c.take<int64_t>(n);
    t.lbits = c.take<int32_t>(n);
    c.off = align_up(c.off, 256);
    t.pool = (int32_t*)((char*)ws + c.off);
    t.pool_slots = 0;
    if (w) *w = t;
    return c.off;
}

// Hash-table slots a vertex of the global-pool path needs: a power of two of
// at least twice its candidate count (load factor at most 1/2).
int pool_bits(int64_t cand)
{
    int b = kHashBits;
    while (((int64_t)1 << b) < 2 * cand) ++b;
    return b;
}

}  // namespace
}  // namespace lt

extern "C" size_t ltsnet_quality_workspace_size(int32_t n, int64_t nnz_graph)
{
    if (n < 1 || nnz_graph < 0) return 0;
    // the largest candidate count is at most deg(v) + nnz <= n + nnz
    const int64_t slots = (int64_t)1 << lt::pool_bits((int64_t)n + nnz_graph);
    return lt::quality_carve(nullptr, n, nullptr) + (size_t)slots * sizeof(int32_t);
}

extern "C" ltsnet_status ltsnet_neighbourhood_preservation(const int64_t* row_ptr, const int32_t* col, int32_t n,
                                                           const float* Y, int32_t* ball, int32_t* common,
                                                           double* np_out, void* ws, size_t ws_bytes,
                                                           ltsnet_stream stream)
{
    using namespace lt;
    if (n < 1 || !row_ptr || !col || !Y || !np_out || !ws) return LTSNET_ERR_INVALID_ARG;
    const size_t fixed = quality_carve(nullptr, n, nullptr);
    if (((uintptr_t)ws & 255) || ws_bytes < fixed) return LTSNET_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    QualityWs w;
    quality_carve(ws, n, &w);
    w.pool_slots = (int64_t)((ws_bytes - fixed) / sizeof(int32_t));
    int32_t* bout = ball ? ball : w.ball;
    int32_t* cout_ = common ? common : w.common;
    const int32_t G = grid_side(n);
    const size_t cells = (size_t)G * G;
    const float2* Y2 = (const float2*)Y;
    QualityScal init{};
    init.lo_ord[0] = init.lo_ord[1] = 0x7fffffff;
    init.hi_ord[0] = init.hi_ord[1] = (int32_t)0x80000000;
    LT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StatusBlock), s));
    LT_CUDA(cudaMemcpyAsync(w.sc, &init, sizeof(QualityScal), cudaMemcpyHostToDevice, s));
    LT_CUDA(cudaMemsetAsync(w.cnt, 0, sizeof(int32_t) * cells, s));
    k_q_bounds<<<kQBlocks, kQThreads, 0, s>>>(Y2, n, w.sc);
    k_q_grid<<<1, 1, 0, s>>>(w.sc, n, G);
    k_q_count<<<kQBlocks, kQThreads, 0, s>>>(Y2, n, w.sc, w.cnt, w.cell);
    k_q_scan<<<1, 1024, 0, s>>>(w.cnt, (int32_t)cells, w.start, w.cursor);
    k_q_scatter<<<kQBlocks, kQThreads, 0, s>>>(Y2, n, w.cell, w.cursor, w.sid, w.sy);
    k_q_sat_rows<<<(G + 127) / 128, 128, 0, s>>>(w.cnt, G, w.sat);
    k_q_sat_cols<<<(G + 127) / 128, 128, 0, s>>>(G, w.sat);
    count_launches(7);
    LT_CHECK_LAUNCH();
    NpArgs A{row_ptr, col, n, Y2, w.sc, w.start, w.sat, w.sid, w.sy, bout, cout_, w.st};
    k_np<<<num_sms() * 6, kNpWarps * 32, 0, s>>>(A, w.sc, w.lv, w.lcand);
    count_launches(1);
    LT_CHECK_LAUNCH();
    // the vertices whose balls go to the global pool, in vertex order, in
    // batches whose tables fit the pool together
    QualityScal hs_sc;
    LT_CUDA(cudaMemcpyAsync(&hs_sc, w.sc, sizeof(QualityScal), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    const int32_t nl = hs_sc.nlarge;
    if (nl > 0) {
        std::vector<int32_t> lv(nl);
        std::vector<int64_t> lc(nl);
        LT_CUDA(cudaMemcpyAsync(lv.data(), w.lv, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
        LT_CUDA(cudaMemcpyAsync(lc.data(), w.lcand, sizeof(int64_t) * nl, cudaMemcpyDeviceToHost, s));
        LT_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> ord(nl);
        for (int32_t i = 0; i < nl; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return lv[x] < lv[y]; });
        std::vector<int32_t> bv(nl), bb(nl);
        std::vector<int64_t> bo(nl);
        int64_t peak = 0;
        for (int32_t i = 0; i < nl; ++i) {
            bv[i] = lv[ord[i]];
            bb[i] = pool_bits(lc[ord[i]]);
            if (bb[i] > 30 || ((int64_t)1 << bb[i]) > w.pool_slots) return LTSNET_ERR_WORKSPACE;
        }
        // batch boundaries and offsets within a batch
        std::vector<int32_t> cut{0};
        int64_t used = 0;
        for (int32_t i = 0; i < nl; ++i) {
            const int64_t sz = (int64_t)1 << bb[i];
            if (used + sz > w.pool_slots) {
                cut.push_back(i);
                used = 0;
            }
            bo[i] = used;
            used += sz;
            peak = std::max(peak, used);
        }
        cut.push_back(nl);
        LT_CUDA(cudaMemsetAsync(w.pool, 0xFF, sizeof(int32_t) * (size_t)peak, s));
        for (size_t q = 0; q + 1 < cut.size(); ++q) {
            const int32_t i0 = cut[q], cnt = cut[q + 1] - cut[q];
            LT_CUDA(cudaMemcpyAsync(w.lv, bv.data() + i0, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s));
            LT_CUDA(cudaMemcpyAsync(w.lcand, bo.data() + i0, sizeof(int64_t) * cnt, cudaMemcpyHostToDevice, s));
            LT_CUDA(cudaMemcpyAsync(w.lbits, bb.data() + i0, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s));
            const int blocks = std::max(1, std::min(num_sms() * 6, (cnt + kNpWarps - 1) / kNpWarps));
            k_np_large<<<blocks, kNpWarps * 32, 0, s>>>(A, w.lv, w.lcand, w.lbits, cnt, w.pool);
            count_launches(1);
            LT_CHECK_LAUNCH();
        }
    }
    k_np_partial<<<kQBlocks, kQThreads, 0, s>>>(bout, cout_, n, w.part, w.pcnt);
    count_launches(1);
    LT_CHECK_LAUNCH();
    double part[kQBlocks];
    unsigned long long pcnt[kQBlocks];
    StatusBlock hs;
    LT_CUDA(cudaMemcpyAsync(part, w.part, sizeof(part), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaMemcpyAsync(pcnt, w.pcnt, sizeof(pcnt), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    if (hs.code) return (ltsnet_status)hs.code;
    double sum = 0.0;
    unsigned long long k = 0;
    for (int q = 0; q < kQBlocks; ++q) {
        sum += part[q];
        k += pcnt[q];
    }
    *np_out = k ? sum / (double)k : 0.0;
    return LTSNET_OK;
}

extern "C" ltsnet_status ltsnet_stress(const int64_t* row_ptr, const int32_t* col, int32_t n, const float* Y,
                                       const int32_t* sources, int32_t n_sources, double* out, void* ws,
                                       size_t ws_bytes, ltsnet_stream stream)
{
    using namespace lt;
    if (n < 1 || n_sources < 1 || !row_ptr || !col || !Y || !sources || !out || !ws) return LTSNET_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255) || ws_bytes < quality_carve(nullptr, n, nullptr)) return LTSNET_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    QualityWs w;
    quality_carve(ws, n, &w);
    const float2* Y2 = (const float2*)Y;
    LT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StatusBlock), s));
    LT_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(LevelCtl), s));
    LT_CUDA(cudaMemsetAsync(w.acc, 0, sizeof(StressAcc) * kQBlocks, s));
    LevelRunner lr{row_ptr, col, n, w.D, w.q0, w.q1, w.ctl, w.st};
    if (ltsnet_status e = lr.prepare()) return e;
    for (int32_t q = 0; q < n_sources; ++q) {
        LT_CUDA(cudaMemsetAsync(w.D, 0xFF, sizeof(uint16_t) * (size_t)n, s));
        k_stress_seed<<<1, 1, 0, s>>>(sources, q, n, w.D, w.q0, w.ctl, w.st);
        count_launches(1);
        LT_CHECK_LAUNCH();
        LevelCtl h;
        if (ltsnet_status e = lr.run(s, &h)) return e;
        if (h.err) break;
        k_stress_accum<<<kQBlocks, kQThreads, 0, s>>>(w.D, Y2, n, sources, q, w.acc);
        count_launches(1);
        LT_CHECK_LAUNCH();
    }
    StressAcc acc[kQBlocks];
    StatusBlock hs;
    LT_CUDA(cudaMemcpyAsync(acc, w.acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    if (hs.code) return (ltsnet_status)hs.code;
    double s1 = 0.0, s2 = 0.0;
    unsigned long long cnt = 0, skipped = 0;
    for (int q = 0; q < kQBlocks; ++q) {
        s1 += acc[q].s1;
        s2 += acc[q].s2;
        cnt += acc[q].cnt;
        skipped += acc[q].skipped;
    }
    const bool ok = cnt > 0 && s2 > 0.0;
    out[0] = ok ? 1.0 - s1 * s1 / ((double)cnt * s2) : 0.0;
    out[1] = ok ? s1 / s2 : 1.0;
    out[2] = (double)cnt;
    out[3] = (double)skipped;
    return LTSNET_OK;
}
