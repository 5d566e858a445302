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
//                 the oracle), FFT plan and twiddles, fixed-point scales, and
//                 the points per box (per-block hash aggregation, then global
//                 atomics).
//  k_box_scan     box offsets, heavy boxes and their segments.
//  k_box_scatter  local coordinates of the points, in box order.
//  k_box_spread   Lagrange weights x charges summed per box in integers and
//                 written as the FP32 charge grid (bit-identical from run to
//                 run).
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

// Forward DFT of size R in place on v[0..R-1] (e^{-2 pi i rq / R}); the
// radix-3 and radix-5 forms pair the inputs symmetrically so that only the
// real constants cos(2 pi k / R), sin(2 pi k / R) appear.
__device__ __forceinline__ float2 mul_mi(float2 z) { return make_float2(z.y, -z.x); }  // -i z

template <int R>
__device__ __forceinline__ void dft_small(float2* v);

template <>
__device__ __forceinline__ void dft_small<2>(float2* v)
{
    const float2 t = v[1];
    v[1] = csub(v[0], t);
    v[0] = cadd(v[0], t);
}

template <>
__device__ __forceinline__ void dft_small<4>(float2* v)
{
    const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const float2 t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[1] = cadd(t1, t3);
    v[2] = csub(t0, t2);
    v[3] = csub(t1, t3);
}

template <>
__device__ __forceinline__ void dft_small<3>(float2* v)
{
    const float s60 = 0.866025403784438647f;  // sin(2 pi / 3)
    const float2 a = cadd(v[1], v[2]);
    const float2 d = mul_mi(csub(v[1], v[2]));
    const float2 m = make_float2(v[0].x - 0.5f * a.x, v[0].y - 0.5f * a.y);
    v[0] = cadd(v[0], a);
    v[1] = make_float2(m.x + s60 * d.x, m.y + s60 * d.y);
    v[2] = make_float2(m.x - s60 * d.x, m.y - s60 * d.y);
}

template <>
__device__ __forceinline__ void dft_small<5>(float2* v)
{
    const float c1 = 0.309016994374947424f, c2 = -0.809016994374947424f;  // cos(2 pi / 5), cos(4 pi / 5)
    const float s1 = 0.951056516295153572f, s2 = 0.587785252292473129f;   // sin(2 pi / 5), sin(4 pi / 5)
    const float2 a1 = cadd(v[1], v[4]), b1 = mul_mi(csub(v[1], v[4]));
    const float2 a2 = cadd(v[2], v[3]), b2 = mul_mi(csub(v[2], v[3]));
    const float2 m1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    const float2 m2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    const float2 n1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
    const float2 n2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(m1, n1);
    v[4] = csub(m1, n1);
    v[2] = cadd(m2, n2);
    v[3] = csub(m2, n2);
}

// ---- in-place FFTs of interleaved line batches ----------------------------
constexpr int kIpThreads = 512;  // threads of the in-place kernels (128 registers for two stages at once)

// nl lines of length L held interleaved in shared memory, element t of line
// l at X[t * ld + l] (ld = nl rounded up to odd, so that both a walk along a
// line and a walk across lines hit distinct banks).  Decimation in frequency
// in place takes natural order to the digit-reversed order of the radix
// sequence; decimation in time with the stages reversed takes that order back
// to natural order.  A convolution therefore needs no permutation pass: the
// products are formed in digit-reversed order, where the position p holds
// frequency drev[p].
//
// Stage k (radix R, span N = R m): butterfly (b, j), b < L / N, j < m, on the
// positions b N + j + r m.  DIF: R-point DFT, then multiply output q by
// e^{-2 pi i j q / N}.  DIT: multiply input r by e^{-2 pi i j r / N}, then the
// R-point DFT.  The twiddle of exponent j q (L / N) is tw[j q ts].
struct LinePlan {
    int32_t L, nst;
    int32_t R[kMaxRadix];
    int32_t m[kMaxRadix];
    uint32_t mg[kMaxRadix];  // floor(2^32 / m) + 1: b = umulhi(beta, mg) exactly for beta, m < 2^12
    int32_t ts[kMaxRadix];
    int32_t np;                // register passes: stage ps[k], and ps[k] + 1 when pp[k]
    int32_t ps[kMaxRadix];
    int32_t pp[kMaxRadix];
};

// Thread 0 fills the plan from the grid's radix sequence; the caller syncs.
__device__ __forceinline__ void make_line_plan(const GridDev& g, LinePlan& pl)
{
    if (threadIdx.x != 0) return;
    pl.L = g.L;
    pl.nst = g.nst;
    int N = g.L;
    for (int k = 0; k < g.nst; ++k) {
        const int R = g.radix[k];
        const int m = N / R;
        pl.R[k] = R;
        pl.m[k] = m;
        pl.mg[k] = m > 1 ? (uint32_t)(4294967296ull / (unsigned)m) + 1u : 0u;
        pl.ts[k] = g.L / N;
        N = m;
    }
    // stages st, st + 1 share one register pass unless their product is above
    // 16 or the first is 5 (registers at 1024 threads)
    int np = 0;
    for (int st = 0; st < g.nst;) {
        const bool pair = st + 1 < g.nst && g.radix[st] * g.radix[st + 1] <= 16 && g.radix[st] != 5;
        pl.ps[np] = st;
        pl.pp[np] = pair ? 1 : 0;
        ++np;
        st += pair ? 2 : 1;
    }
    pl.np = np;
}

// drev[p] = the frequency that DIF leaves at position p; pos_of is its
// inverse.  Position p has digits q_k = (p / m_k) mod R_k and frequency
// sum_k q_k R_1 ... R_{k-1}.
__device__ __forceinline__ void make_digit_tables(const LinePlan& pl, uint16_t* drev, uint16_t* pos_of)
{
    for (int p = threadIdx.x; p < pl.L; p += blockDim.x) {
        int k = 0, place = 1;
        for (int st = 0; st < pl.nst; ++st) {
            const int q = (p / pl.m[st]) % pl.R[st];
            k += q * place;
            place *= pl.R[st];
        }
        drev[p] = (uint16_t)k;
        if (pos_of) pos_of[k] = (uint16_t)p;
    }
}

template <int R, bool DIT>
__device__ __forceinline__ void ip_stage(float2* X, int ld, int nl, const LinePlan& pl, int st, const float2* tw,
                                         int tl, int tb, int nbp)
{
    const int m = pl.m[st];
    const uint32_t mg = pl.mg[st];
    const int ts = pl.ts[st];
    const int nbf = pl.L / R;
    for (int beta = tb; beta < nbf; beta += nbp) {
        const int b = m > 1 ? (int)__umulhi((uint32_t)beta, mg) : beta;
        const int j = beta - b * m;
        float2* x = X + (int64_t)(b * R * m + j) * ld + tl;
        const int step = m * ld;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[r * step];
        if (DIT) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * ts]);
        }
        dft_small<R>(v);
        if (!DIT) {
#pragma unroll
            for (int q = 1; q < R; ++q) v[q] = cmul(v[q], tw[j * q * ts]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) x[q * step] = v[q];
    }
}

// Stages st and st + 1 in registers: the R1 R2 positions b N + j' + r1 m +
// r2 m2 (N = R1 m, m = R2 m2, j' < m2) are closed under both stages.  DIF:
// stage st over r1 for each r2 (j = j' + r2 m2), then stage st + 1 over r2 for
// each output q1 of the first.  DIT: the same two stages transposed, in the
// reverse order.
template <int R1, int R2, bool DIT>
__device__ __forceinline__ void ip_stage2(float2* X, int ld, const LinePlan& pl, int st, const float2* tw, int tl,
                                          int tb, int nbp)
{
    const int m = pl.m[st], m2 = pl.m[st + 1];
    const uint32_t mg2 = pl.mg[st + 1];
    const int ts1 = pl.ts[st], ts2 = pl.ts[st + 1];
    const int nb = pl.L / (R1 * R2);
    for (int beta = tb; beta < nb; beta += nbp) {
        const int b = m2 > 1 ? (int)__umulhi((uint32_t)beta, mg2) : beta;
        const int jp = beta - b * m2;
        float2* x = X + (int64_t)(b * R1 * m + jp) * ld + tl;
        float2 v[R1][R2];
#pragma unroll
        for (int r1 = 0; r1 < R1; ++r1)
#pragma unroll
            for (int r2 = 0; r2 < R2; ++r2) v[r1][r2] = x[(int64_t)(r1 * m + r2 * m2) * ld];
        if (!DIT) {
#pragma unroll
            for (int r2 = 0; r2 < R2; ++r2) {
                float2 u[R1];
#pragma unroll
                for (int r1 = 0; r1 < R1; ++r1) u[r1] = v[r1][r2];
                dft_small<R1>(u);
                const int j = jp + r2 * m2;
#pragma unroll
                for (int q1 = 0; q1 < R1; ++q1) v[q1][r2] = q1 ? cmul(u[q1], tw[j * q1 * ts1]) : u[0];
            }
#pragma unroll
            for (int q1 = 0; q1 < R1; ++q1) {
                dft_small<R2>(v[q1]);
#pragma unroll
                for (int q2 = 1; q2 < R2; ++q2) v[q1][q2] = cmul(v[q1][q2], tw[jp * q2 * ts2]);
            }
        } else {
#pragma unroll
            for (int r1 = 0; r1 < R1; ++r1) {
#pragma unroll
                for (int r2 = 1; r2 < R2; ++r2) v[r1][r2] = cmul(v[r1][r2], tw[jp * r2 * ts2]);
                dft_small<R2>(v[r1]);
            }
#pragma unroll
            for (int q2 = 0; q2 < R2; ++q2) {
                const int j = jp + q2 * m2;
                float2 u[R1];
#pragma unroll
                for (int r1 = 0; r1 < R1; ++r1) u[r1] = r1 ? cmul(v[r1][q2], tw[j * r1 * ts1]) : v[0][q2];
                dft_small<R1>(u);
#pragma unroll
                for (int q1 = 0; q1 < R1; ++q1) v[q1][q2] = u[q1];
            }
        }
#pragma unroll
        for (int r1 = 0; r1 < R1; ++r1)
#pragma unroll
            for (int r2 = 0; r2 < R2; ++r2) x[(int64_t)(r1 * m + r2 * m2) * ld] = v[r1][r2];
    }
}

// One pass over the lines: stages st (and st + 1 when pair) of the plan.
template <bool DIT>
__device__ __forceinline__ void ip_pass(float2* X, int ld, int nl, const LinePlan& pl, int st, bool pair,
                                        const float2* tw, int tl, int tb, int nbp)
{
    if (!pair) {
        switch (pl.R[st]) {
            case 4: ip_stage<4, DIT>(X, ld, nl, pl, st, tw, tl, tb, nbp); break;
            case 2: ip_stage<2, DIT>(X, ld, nl, pl, st, tw, tl, tb, nbp); break;
            case 3: ip_stage<3, DIT>(X, ld, nl, pl, st, tw, tl, tb, nbp); break;
            default: ip_stage<5, DIT>(X, ld, nl, pl, st, tw, tl, tb, nbp); break;
        }
        return;
    }
    switch (pl.R[st] * 8 + pl.R[st + 1]) {
        case 4 * 8 + 4: ip_stage2<4, 4, DIT>(X, ld, pl, st, tw, tl, tb, nbp); break;
        case 4 * 8 + 2: ip_stage2<4, 2, DIT>(X, ld, pl, st, tw, tl, tb, nbp); break;
        case 4 * 8 + 3: ip_stage2<4, 3, DIT>(X, ld, pl, st, tw, tl, tb, nbp); break;
        case 2 * 8 + 3: ip_stage2<2, 3, DIT>(X, ld, pl, st, tw, tl, tb, nbp); break;
        case 2 * 8 + 5: ip_stage2<2, 5, DIT>(X, ld, pl, st, tw, tl, tb, nbp); break;
        case 3 * 8 + 3: ip_stage2<3, 3, DIT>(X, ld, pl, st, tw, tl, tb, nbp); break;
        default: ip_stage2<3, 5, DIT>(X, ld, pl, st, tw, tl, tb, nbp); break;  // 3 x 5
    }
}

// Forward DFT of the nl interleaved lines in place: DIF (natural order in,
// digit-reversed out) or DIT (digit-reversed in, natural out), in the
// plan's register passes (DIT runs them in reverse).  All threads of the
// block call it; it ends with a barrier.
template <bool DIT>
__device__ void ip_fft(float2* X, int ld, int nl, const LinePlan& pl, const float2* tw)
{
    const int nbp = (int)blockDim.x / nl;
    const int tl = (int)threadIdx.x % nl;
    const int tb = (int)threadIdx.x / nl;
    const bool on = tb < nbp;
    for (int k = 0; k < pl.np; ++k) {
        const int q = DIT ? pl.np - 1 - k : k;
        if (on) ip_pass<DIT>(X, ld, nl, pl, pl.ps[q], pl.pp[q] != 0, tw, tl, tb, nbp);
        __syncthreads();
    }
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
    g.rh = __frcp_rn(g.h);
    g.rs = __frcp_rn(g.s);
    g.c = __fmul_rn(0.5f, __fadd_rn(lo, hi));
    g.I = I;
    g.P = P;
    g.M = I * P;
    g.L = 2 * g.M;
    int r = g.L, k = 0;
    while (r % 4 == 0) { g.radix[k++] = 4; r /= 4; }
    while (r % 2 == 0) { g.radix[k++] = 2; r /= 2; }
    while (r % 3 == 0) { g.radix[k++] = 3; r /= 3; }
    while (r % 5 == 0) { g.radix[k++] = 5; r /= 5; }
    g.nst = k;
    // node-local charges (1, ex, ey, ex^2 + ey^2) with |e| <= P in node units,
    // Lagrange weight products <= 8 for P <= 5: 64-bit fixed point with room
    // for the sum over all n points
    const double qb[4] = {1.0, (double)P, (double)P, 2.0 * P * P};
    for (int c = 0; c < 4; ++c) {
        int ex;
        frexp((double)n * 8.0 * qb[c], &ex);
        g.fx[c] = ldexpf(1.0f, 62 - ex);
        g.ifx[c] = ldexpf(1.0f, ex - 62);
    }
    // Per-point 32-bit quantisation of the warp-summed (heavy) boxes: bounds
    // of |w|, |w e|, |w e|, |w |e|^2| over local coordinates in
    // [-0.05, P + 0.05] (tensor Lagrange weights w, offsets e from the nodes),
    // scaled to at most 2^22 so that the round-to-integer by adding 1.5 * 2^23
    // is exact and kSeg points sum below 2^31.
    const float hb[4][4] = {{2.41f, 3.91f, 6.20f, 14.26f},
                            {1.33f, 4.30f, 9.61f, 33.2f},
                            {1.33f, 4.30f, 9.61f, 33.2f},
                            {4.10f, 13.4f, 49.0f, 169.1f}};
    for (int c = 0; c < 4; ++c) {
        int ex;
        frexpf(4194304.0f / hb[c][P - 2], &ex);
        g.hf[c] = ldexpf(1.0f, ex - 1);
        g.ihf[c] = ldexpf(1.0f, 1 - ex);
    }
}

// Points are taken in tiles of kBoxTile consecutive indices per block.  The
// boxes a tile touches are aggregated in a shared-memory hash table (at most
// kBoxTile keys in 2 kBoxTile slots, linear probing), so a box that holds
// most of the points receives one global atomic per tile instead of one per
// warp.
constexpr int kBoxThreads = 256;
constexpr int kBoxRounds = 4;
constexpr int kBoxTile = kBoxThreads * kBoxRounds;
constexpr int kBoxHash = 2 * kBoxTile;

struct BoxHash {
    int key[kBoxHash];
    int val[kBoxHash];
    int base[kBoxHash];
};

__device__ __forceinline__ void box_hash_clear(BoxHash& H)
{
    for (int i = threadIdx.x; i < kBoxHash; i += blockDim.x) {
        H.key[i] = -1;
        H.val[i] = 0;
    }
}

// Slot of `box` (inserted if absent); the table never holds more than half
// its slots, so the probe ends within kBoxHash steps.
__device__ __forceinline__ int box_hash_slot(BoxHash& H, int box)
{
    int slot = (int)(((unsigned)box * 2654435761u) >> 21) & (kBoxHash - 1);
    for (int k = 0; k < kBoxHash; ++k) {
        const int old = atomicCAS(&H.key[slot], -1, box);
        if (old == -1 || old == box) return slot;
        slot = (slot + 1) & (kBoxHash - 1);
    }
    return -1;
}

// Points per box, in tiles of kBoxTile consecutive points per block: the
// boxes a tile touches are aggregated in the shared-memory hash table and
// added to bcnt.  count_prefetch loads the block's first tile and clears the
// table (it needs no grid, so it runs while the grid is being derived);
// count_tiles then counts that tile and the block's later ones.
__device__ __forceinline__ void count_prefetch(const float2* __restrict__ Y, int32_t n, BoxHash& H,
                                               float2 (&pts)[kBoxRounds])
{
    const int64_t ntiles = ((int64_t)n + kBoxTile - 1) / kBoxTile;
    if ((int64_t)blockIdx.x >= ntiles) return;
#pragma unroll
    for (int r = 0; r < kBoxRounds; ++r) {
        const int64_t i = (int64_t)blockIdx.x * kBoxTile + r * kBoxThreads + threadIdx.x;
        pts[r] = i < n ? Y[i] : make_float2(0.f, 0.f);
    }
    box_hash_clear(H);
}

__device__ __forceinline__ void count_tiles(const float2* __restrict__ Y, int32_t n, float lo, float h, float rh,
                                            int I, int32_t* __restrict__ bcnt, BoxHash& H,
                                            float2 (&pts)[kBoxRounds])
{
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = ((int64_t)n + kBoxTile - 1) / kBoxTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (tile != (int64_t)blockIdx.x) {
            box_hash_clear(H);
#pragma unroll
            for (int r = 0; r < kBoxRounds; ++r) {
                const int64_t i = tile * kBoxTile + r * kBoxThreads + threadIdx.x;
                pts[r] = i < n ? Y[i] : make_float2(0.f, 0.f);
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < kBoxRounds; ++r) {
            const int64_t i = tile * kBoxTile + r * kBoxThreads + threadIdx.x;
            const int box = i < n ? box_of_r(pts[r].y, lo, h, rh, I) * I + box_of_r(pts[r].x, lo, h, rh, I) : -1;
            const unsigned peers = __match_any_sync(FULL, box);
            if (box >= 0 && lane == __ffs(peers) - 1) {
                const int slot = box_hash_slot(H, box);
                if (slot >= 0) atomicAdd(&H.val[slot], __popc(peers));
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kBoxHash; k += blockDim.x)
            if (H.key[k] >= 0) atomicAdd(&bcnt[H.key[k]], H.val[k]);
        __syncthreads();
    }
}

// Grid of this iteration (every block derives the same grid from the bounds;
// block 0 publishes it), FFT twiddles, and -- unless the plain atomic spread
// is in use -- the points per box, aggregated per tile of kBoxTile points in
// a shared-memory hash table and added to bcnt, which the previous
// iteration's last kernel (or the workspace reset) left zero.
__device__ __forceinline__ void k_setup_body(const int32_t* __restrict__ bounds_cur,
                                                       int32_t* __restrict__ bounds_next, GridDev* G,
                                                       float2* __restrict__ tw, const float2* __restrict__ Y,
                                                       int32_t* __restrict__ bcnt, int32_t n, float bwm, int min_boxes,
                                                       int max_boxes, int P, int count)
{
    __shared__ GridDev g;
    __shared__ BoxHash H;
    // the first tile's points and the hash table are made ready while
    // thread 0 derives the grid
    float2 pts[kBoxRounds];
    if (count) count_prefetch(Y, n, H, pts);
    if (threadIdx.x == 0) compute_grid(bounds_cur, bwm, min_boxes, max_boxes, P, n, g);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        G->lo = g.lo; G->hi = g.hi; G->ext = g.ext; G->h = g.h; G->s = g.s; G->c = g.c;
        G->rh = g.rh; G->rs = g.rs;
        G->I = g.I; G->M = g.M; G->L = g.L; G->P = g.P;
        G->nst = g.nst;
        for (int i = 0; i < kMaxRadix; ++i) G->radix[i] = i < g.nst ? g.radix[i] : 0;
        for (int c = 0; c < 4; ++c) {
            G->fx[c] = g.fx[c];
            G->ifx[c] = g.ifx[c];
            G->hf[c] = g.hf[c];
            G->ihf[c] = g.ihf[c];
        }
        G->ticket = 0;
        G->imax = max(G->imax, g.I);
        G->nheavy = 0;
        G->nitems = 0;
        G->scan_ticket = 0;
        bounds_next[0] = f2ord(INFINITY);
        bounds_next[1] = f2ord(-INFINITY);
    }
    if (count) count_tiles(Y, n, g.lo, g.h, g.rh, g.I, bcnt, H, pts);
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
}

__global__ void __launch_bounds__(kBoxThreads) k_setup(const int32_t* __restrict__ bounds_cur,
                                                       int32_t* __restrict__ bounds_next, GridDev* G,
                                                       float2* __restrict__ tw, const float2* __restrict__ Y,
                                                       int32_t* __restrict__ bcnt, int32_t n, float bwm, int min_boxes,
                                                       int max_boxes, int P, int count)
{
    k_setup_body(bounds_cur, bounds_next, G, tw, Y, bcnt, n, bwm, min_boxes, max_boxes, P, count);
}

// ---- deterministic spread: box sort, then integer sums per box ----
// The Lagrange nodes a point feeds are those of its own box, so every node's
// charges are sums over one box's points.  The points are counted per box,
// the counts scanned, and the points scattered into box order with their
// local coordinates.  Then every box is summed in integers -- a thread per
// (box, node row) for boxes of at most kLightMax points, warps over segments
// of kSeg points for the rest -- so the sums do not depend on the order of
// the points within a box.  Every node's final FP32 charges are written once
// per iteration, with no atomics on the grid and no clearing pass, and the
// grid is bit-identical from run to run.

constexpr int kScanBlock = 256;   // boxes per chunk of the box scan (one per thread)
constexpr int kMaxScanChunks = 4096;  // max_boxes <= 1024
constexpr int kLightMax = 8;      // boxes with more points are summed by warps
constexpr int kSeg = 256;         // points per warp work item of a heavy box

// Box offsets, in chunks of kScanBlock boxes (one per thread): chunk-local
// exclusive offsets into bcur (the scatter cursors), chunk totals into btot,
// and, by the last block to finish, the exclusive scan of the totals into
// bpre; a box's points start at bpre[box / kScanBlock] + (local offset).
// Boxes with more than kLightMax points are listed in heavy[0 .. G->nheavy),
// and their segments of kSeg points in items[0 .. G->nitems) as (heavy index,
// segment).
constexpr int kScanThreads = kScanBlock;

__device__ __forceinline__ int block_exclusive_scan256(int v, int* wsum, int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int x = lane < (kScanThreads >> 5) ? wsum[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += u;
        }
        if (lane < (kScanThreads >> 5)) wsum[lane] = xi - x;
        if (lane == 31) wsum[32] = xi;
    }
    __syncthreads();
    const int r = wsum[w] + inc - v;
    *total = wsum[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void list_heavy(GridDev* __restrict__ G, int b, int v, int32_t* __restrict__ heavy,
                                           int2* __restrict__ items)
{
    const bool hv = v > kLightMax;
    const unsigned hm = __ballot_sync(FULL, hv);
    if (!hm) return;
    const int lane = threadIdx.x & 31, leader = __ffs(hm) - 1;
    const int nseg = hv ? (v + kSeg - 1) / kSeg : 0;
    int inc = nseg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += u;
    }
    const int nall = __shfl_sync(FULL, inc, 31);
    int hbase = 0, ibase = 0;
    if (lane == leader) {
        hbase = atomicAdd(&G->nheavy, __popc(hm));
        ibase = atomicAdd(&G->nitems, nall);
    }
    hbase = __shfl_sync(FULL, hbase, leader);
    ibase = __shfl_sync(FULL, ibase, leader);
    if (hv) heavy[hbase + __popc(hm & lanemask_lt())] = b;
    for (int k0 = 0; k0 < nall; k0 += 32) {
        const int k = k0 + lane;
        int owner = 0;  // first lane whose inclusive segment count exceeds k (binary search)
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int probe = __shfl_sync(FULL, inc, owner + step - 1);
            if (probe <= k) owner += step;
        }
        owner = min(owner, 31);
        const int ex = __shfl_sync(FULL, inc - nseg, owner);
        if (k < nall) items[ibase + k] = make_int2(hbase + __popc(hm & ((1u << owner) - 1u)), k - ex);
    }
}

__device__ __forceinline__ void k_box_scan_body(GridDev* __restrict__ G, const int32_t* __restrict__ bcnt,
                                                           int32_t* __restrict__ bcur, int32_t* __restrict__ btot,
                                                           int32_t* __restrict__ bpre, int32_t* __restrict__ heavy,
                                                           int2* __restrict__ items)
{
    __shared__ int wsum[33];
    __shared__ bool last;
    const int NB = G->I * G->I;
    const int nchunks = (NB + kScanBlock - 1) / kScanBlock;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int b = c * kScanBlock + threadIdx.x;
        const int v = b < NB ? bcnt[b] : 0;
        int tot;
        const int ex = block_exclusive_scan256(v, wsum, &tot);
        if (b < NB) bcur[b] = ex;
        list_heavy(G, b, v, heavy, items);
        if (threadIdx.x == 0) btot[c] = tot;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&G->scan_ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive scan of up to kMaxScanChunks chunk totals, 16 per thread
    constexpr int kPer = kMaxScanChunks / kScanThreads;
    int v[kPer], t = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int c = kPer * threadIdx.x + k;
        v[k] = c < nchunks ? ((volatile int32_t*)btot)[c] : 0;
        t += v[k];
    }
    int all;
    int ex = block_exclusive_scan256(t, wsum, &all);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int c = kPer * threadIdx.x + k;
        if (c < nchunks) bpre[c] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) G->scan_ticket = 0;
}

__global__ void __launch_bounds__(kScanThreads) k_box_scan(GridDev* __restrict__ G, const int32_t* __restrict__ bcnt,
                                                           int32_t* __restrict__ bcur, int32_t* __restrict__ btot,
                                                           int32_t* __restrict__ bpre, int32_t* __restrict__ heavy,
                                                           int2* __restrict__ items)
{
    k_box_scan_body(G, bcnt, bcur, btot, bpre, heavy, items);
}

// Same tiles and hash table as the counting in k_setup: each box a tile touches reserves
// its range once (one global atomic), and the tile's points of that box take
// consecutive places in it.
__device__ __forceinline__ void k_box_scatter_body(const float2* __restrict__ Y, int32_t n,
                                                             const GridDev* __restrict__ G,
                                                             int32_t* __restrict__ bcur,
                                                             const int32_t* __restrict__ bpre,
                                                             float2* __restrict__ su)
{
    __shared__ BoxHash H;
    const float lo = G->lo, h = G->h, s = G->s, rh = G->rh, rs = G->rs;
    const int I = G->I, P = G->P;
    const int lane = threadIdx.x & 31;
    const unsigned ltm = lanemask_lt();
    const int64_t ntiles = ((int64_t)n + kBoxTile - 1) / kBoxTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        box_hash_clear(H);
        __syncthreads();
        float2 pt[kBoxRounds];
        int slot[kBoxRounds], off[kBoxRounds], bxy[kBoxRounds];
#pragma unroll
        for (int r = 0; r < kBoxRounds; ++r) {
            const int64_t i = tile * kBoxTile + r * kBoxThreads + threadIdx.x;
            int box = -1, bx = 0, by = 0;
            pt[r] = make_float2(0.f, 0.f);
            if (i < n) {
                pt[r] = Y[i];
                bx = box_of_r(pt[r].x, lo, h, rh, I);
                by = box_of_r(pt[r].y, lo, h, rh, I);
                box = by * I + bx;
            }
            bxy[r] = (by << 16) | bx;
            const unsigned peers = __match_any_sync(FULL, box);
            const int leader = __ffs(peers) - 1;
            int sl = -1, o = 0;
            if (box >= 0 && lane == leader) {
                sl = box_hash_slot(H, box);
                if (sl >= 0) o = atomicAdd(&H.val[sl], __popc(peers));
            }
            sl = __shfl_sync(FULL, sl, leader);
            o = __shfl_sync(FULL, o, leader);
            slot[r] = box >= 0 ? sl : -1;
            off[r] = o + __popc(peers & ltm);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kBoxHash; k += blockDim.x) {
            const int key = H.key[k];
            if (key >= 0) H.base[k] = bpre[key / kScanBlock] + atomicAdd(&bcur[key], H.val[k]);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kBoxRounds; ++r) {
            if (slot[r] < 0) continue;
            const int bx = bxy[r] & 0xffff, by = bxy[r] >> 16;
            su[H.base[slot[r]] + off[r]] =
                make_float2(local_u(pt[r].x, lo, s, rs, P * bx), local_u(pt[r].y, lo, s, rs, P * by));
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBoxThreads) k_box_scatter(const float2* __restrict__ Y, int32_t n,
                                                             const GridDev* __restrict__ G,
                                                             int32_t* __restrict__ bcur,
                                                             const int32_t* __restrict__ bpre,
                                                             float2* __restrict__ su)
{
    k_box_scatter_body(Y, n, G, bcur, bpre, su);
}

// |v| < 2^63 to FP32 with integer operations only (two roundings, relative
// error below 2^-22), then scaled by the power of two 1/fx.
__device__ __forceinline__ float fix_to_float(long long v, float ifx)
{
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const float f = __fmaf_rn((float)(unsigned)(a >> 32), 4294967296.0f, (float)(unsigned)a);
    return (v < 0 ? -f : f) * ifx;
}

// Charges of one point on node row bb of its box, added to the fixed-point
// sums ra[a][0..3] of the row's P nodes: (w, w ex, w ey, w |e|^2) with w the
// tensor Lagrange weight and e the offset from the node in node spacings.
template <int P>
__device__ __forceinline__ void add_point_row(float2 u, int bb, const float* fx, long long (*ra)[4])
{
    float wx[P];
    lagrange<P>(u.x, wx);
    const float wyb = lagrange_one<P>(u.y, bb);
    const float ey = u.y - ((float)bb + 0.5f);
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const float w = wx[a] * wyb;
        const float ex = u.x - ((float)a + 0.5f);
        ra[a][0] += f2ll_rn(w * fx[0]);
        ra[a][1] += f2ll_rn((w * ex) * fx[1]);
        ra[a][2] += f2ll_rn((w * ey) * fx[2]);
        ra[a][3] += f2ll_rn((w * (ex * ex + ey * ey)) * fx[3]);
    }
}

// Charges of one point on node row bb, quantised to integers of the scale
// hf (|value| * hf < 2^22) by adding 1.5 * 2^23 -- the sum is then exactly
// the rounded value plus that constant, whose bit pattern is accumulated and
// removed once per lane at the end.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr unsigned kMagicBits = 0x4B400000u;

template <int P>
__device__ __forceinline__ void add_point_row_q(float2 u, int bb, const float* hf, unsigned (*ra)[4])
{
    float wx[P];
    lagrange<P>(u.x, wx);
    const float wyb = lagrange_one<P>(u.y, bb);
    const float ey = u.y - ((float)bb + 0.5f);
    const float ey2 = ey * ey;
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const float w = wx[a] * wyb;
        const float ex = u.x - ((float)a + 0.5f);
        ra[a][0] += __float_as_uint(__fmaf_rn(w, hf[0], kMagic));
        ra[a][1] += __float_as_uint(__fmaf_rn(w * ex, hf[1], kMagic));
        ra[a][2] += __float_as_uint(__fmaf_rn(w * ey, hf[2], kMagic));
        ra[a][3] += __float_as_uint(__fmaf_rn(w * __fmaf_rn(ex, ex, ey2), hf[3], kMagic));
    }
}

// Totals of NV (16 or 32) per-lane values over the warp by reduce-scatter:
// each level halves the values a lane holds, so lane l ends with the total
// of value l (NV = 32) or l >> 1 (NV = 16, both lanes of a pair) after NV - 1
// shuffles instead of 5 NV.  Sums modulo 2^32, so the order of the additions
// does not matter.
template <int NV>
__device__ __forceinline__ unsigned warp_reduce_scatter(unsigned (&v)[NV], int lane)
{
#pragma unroll
    for (int h = NV / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const unsigned send = up ? v[i] : v[i + h];
            const unsigned keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, o);
        }
    }
    if (NV == 16) v[0] += __shfl_xor_sync(FULL, v[0], 1);
    return v[0];
}

// The charge grid from the box-sorted points, every node written once.
// (1) Boxes of more than kLightMax points, one warp per segment of kSeg
// points (held in registers), node row by node row: the lanes sum strided
// points in 32-bit integers and the sums are reduced across the warp
// (reduce-scatter).  A box of one segment is written
// directly; for the others the segments add their sums to the box's 64-bit
// accumulator, and the warp that finishes last (a ticket per box) converts
// it, writes the box's nodes and clears the accumulator and the ticket for
// the next iteration.  (2) The other boxes, one thread per (box row, node
// row, box column) -- consecutive threads write consecutive nodes of a grid
// row -- with exact 64-bit fixed-point sums (empty boxes write zeros).
// Integer sums make the grid independent of the order of the points within
// a box and of which warp finishes when.
template <int P>
__device__ __forceinline__ void k_box_spread_body(const float2* __restrict__ su, const int32_t* __restrict__ bcnt,
                                                    const int32_t* __restrict__ bcur,
                                                    const int32_t* __restrict__ bpre,
                                                    const int32_t* __restrict__ heavy,
                                                    const int2* __restrict__ items, long long* __restrict__ hacc,
                                                    int32_t* __restrict__ hticket, const GridDev* __restrict__ G,
                                                    float4* __restrict__ wflt)
{
    const int I = G->I, M = G->M;
    const int nit = G->nitems;
    float hf[4], ihf[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        hf[q] = G->hf[q];
        ihf[q] = G->ihf[q];
    }
    const int lane = threadIdx.x & 31;
    const int nw = (int)(gridDim.x * blockDim.x) >> 5;
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    for (int base = wid; base < nit; base += nw * 32) {
        // The warp's items are base, base + nw, ...: lane j fetches the box,
        // count and first point of the j-th, so that the chain of dependent
        // loads (item, heavy box, count and offsets) is paid once per 32
        // items; the items are then summed one after the other as before.
        int m_hb = 0, m_seg = 0, m_box = 0, m_cnt = 0, m_start = 0;
        {
            const int itj = base + lane * nw;
            if (itj < nit) {
                const int2 item = items[itj];
                m_hb = item.x;
                m_seg = item.y;
                m_box = heavy[m_hb];
                m_cnt = bcnt[m_box];
                m_start = bpre[m_box / kScanBlock] + bcur[m_box] - m_cnt;
            }
        }
        const int nj = min(32, (nit - base + nw - 1) / nw);
        for (int j = 0; j < nj; ++j) {
            const int hb = __shfl_sync(FULL, m_hb, j);
            const int box = __shfl_sync(FULL, m_box, j);
            const int cnt = __shfl_sync(FULL, m_cnt, j);
            const int start = __shfl_sync(FULL, m_start, j);
            const int seg = __shfl_sync(FULL, m_seg, j);
            const int nseg = (cnt + kSeg - 1) / kSeg;
            const int q0 = start + seg * kSeg, q1 = min(start + cnt, q0 + kSeg);
            const int by = box / I, bx = box - by * I;
            // the segment's points, all loads issued before any is used
            float2 pts[kSeg / 32];
#pragma unroll
            for (int k = 0; k < kSeg / 32; ++k) {
                const int q = q0 + lane + 32 * k;
                pts[k] = q < q1 ? su[q] : make_float2(0.f, 0.f);
            }
            const unsigned m = (unsigned)max(0, min(kSeg / 32, (q1 - q0 - lane + 31) / 32));  // points of this lane
            long long* acc = hacc + (int64_t)hb * P * P * 4;
            for (int bb = 0; bb < P; ++bb) {
                unsigned ra[P][4];  // sums modulo 2^32; the true sums are below 2^31
#pragma unroll
                for (int a = 0; a < P; ++a)
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) ra[a][ch] = 0u;
#pragma unroll
                for (int k = 0; k < kSeg / 32; ++k)
                    if ((unsigned)k < m) add_point_row_q<P>(pts[k], bb, hf, ra);
                const unsigned bias = m * kMagicBits;
                // value a * 4 + ch of the row, padded with zeros to NV values
                constexpr int NV = P * 4 <= 16 ? 16 : 32;
                unsigned vals[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) vals[v] = v < P * 4 ? ra[v >> 2][v & 3] - bias : 0u;
                const unsigned tot = warp_reduce_scatter<NV>(vals, lane);
                const int vi = NV == 32 ? lane : lane >> 1;  // the value this lane now holds the total of
                if (nseg == 1) {
                    // node a = lane < P gathers its four moments from their lanes
                    const int a = min(lane, P - 1);
                    unsigned c[4];
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch)
                        c[ch] = __shfl_sync(FULL, tot, NV == 32 ? 4 * a + ch : 2 * (4 * a + ch));
                    if (lane < P)
                        wflt[(int64_t)(by * P + bb) * M + (int64_t)bx * P + lane] =
                            make_float4((float)(int)c[0] * ihf[0], (float)(int)c[1] * ihf[1], (float)(int)c[2] * ihf[2],
                                        (float)(int)c[3] * ihf[3]);
                } else if ((NV == 32 || (lane & 1) == 0) && vi < P * 4 && tot != 0u) {
                    atomicAdd((unsigned long long*)(acc + bb * P * 4 + vi), (unsigned long long)(long long)(int)tot);
                }
            }
            if (nseg == 1) continue;
            __threadfence();
            int last = 0;
            if (lane == 0) last = atomicAdd(&hticket[hb], 1) == nseg - 1;
            last = __shfl_sync(FULL, last, 0);
            if (!last) continue;
            __threadfence();
            if (lane < P * P) {
                const int nb = lane / P, a = lane - nb * P;
                long long* q = acc + lane * 4;
                const long long c0 = __ldcg(q + 0), c1 = __ldcg(q + 1), c2 = __ldcg(q + 2), c3 = __ldcg(q + 3);
                wflt[(int64_t)(by * P + nb) * M + (int64_t)bx * P + a] =
                    make_float4(fix_to_float(c0, ihf[0]), fix_to_float(c1, ihf[1]), fix_to_float(c2, ihf[2]),
                                fix_to_float(c3, ihf[3]));
                q[0] = 0;
                q[1] = 0;
                q[2] = 0;
                q[3] = 0;
            }
            if (lane == 0) hticket[hb] = 0;
        }
    }

    float fx[4], ifx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        fx[q] = G->fx[q];
        ifx[q] = G->ifx[q];
    }
    const int64_t total = (int64_t)I * I * P;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(t % I);
        const int r = (int)(t / I);
        const int by = r / P, bb = r - by * P;
        const int box = by * I + bx;
        const int cnt = bcnt[box];
        if (cnt > kLightMax) continue;
        long long ra[P][4];
#pragma unroll
        for (int a = 0; a < P; ++a)
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) ra[a][ch] = 0;
        const int start = bpre[box / kScanBlock] + bcur[box] - cnt;
        float2 nxt = cnt > 0 ? su[start] : make_float2(0.f, 0.f);
        for (int q = start; q < start + cnt; ++q) {
            const float2 cur = nxt;
            if (q + 1 < start + cnt) nxt = su[q + 1];
            add_point_row<P>(cur, bb, fx, ra);
        }
        float4* dst = wflt + (int64_t)(by * P + bb) * M + (int64_t)bx * P;
#pragma unroll
        for (int a = 0; a < P; ++a)
            dst[a] = make_float4(fix_to_float(ra[a][0], ifx[0]), fix_to_float(ra[a][1], ifx[1]),
                                 fix_to_float(ra[a][2], ifx[2]), fix_to_float(ra[a][3], ifx[3]));
    }
}

template <int P>
__global__ void __launch_bounds__(256) k_box_spread(const float2* __restrict__ su, const int32_t* __restrict__ bcnt,
                                                    const int32_t* __restrict__ bcur,
                                                    const int32_t* __restrict__ bpre,
                                                    const int32_t* __restrict__ heavy,
                                                    const int2* __restrict__ items, long long* __restrict__ hacc,
                                                    int32_t* __restrict__ hticket, const GridDev* __restrict__ G,
                                                    float4* __restrict__ wflt)
{
    k_box_spread_body<P>(su, bcnt, bcur, bpre, heavy, items, hacc, hticket, G, wflt);
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

__device__ __forceinline__ void load_tw(float2* stw, const float2* __restrict__ tw, int L)
{
    for (int t = threadIdx.x; t < L; t += blockDim.x) stw[t] = tw[t];
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
constexpr float kLnScale = 1.0f / 1024.0f;  // ln(eps + d^2) packed beside K1, scaled to K1's magnitude

// Shared-memory carve of the in-place line kernels: twiddles (unless they
// are read from global memory), digit tables, then the line buffer.
struct IpSmem {
    const float2* tw;  // smem copy or the global table
    uint16_t* drev;
    uint16_t* pos_of;  // null unless requested
    float2* X;
    int avail;         // float2 slots left for X
};

__device__ __forceinline__ IpSmem ip_smem(float2* smf, int sm_f2, int L, bool pos_tab, bool tw_smem,
                                          const float2* __restrict__ tw)
{
    IpSmem r;
    const int tab = ((pos_tab ? 2 : 1) * L + 3) / 4;  // uint16 tables in float2 slots
    float2* p = smf;
    if (tw_smem) {
        load_tw(p, tw, L);
        r.tw = p;
        p += L;
    } else {
        r.tw = tw;
    }
    r.drev = (uint16_t*)p;
    r.pos_of = pos_tab ? r.drev + L : nullptr;
    r.X = p + tab;
    r.avail = sm_f2 - (int)(r.X - smf);
    return r;
}

// Kernel spectrum records: for (kx, ky) in [0, H)^2 eight floats
//   a = (K2^, Ke^, K1^, ln^),  b = (D2x, Dex, D2y, Dey)
// (D = Im of the odd kernels' spectra, scaled like the even ones by 1/L^2).
// The kernels depend on |dx| and |dy| only (times dx or dy for the odd ones),
// so D?y(kx, ky) = D?x(ky, kx); the even spectra and D?x are even in ky and
// D?y is odd in ky.  kc_at unfolds ky in [0, L).
__device__ __forceinline__ void kc_at(const float4* __restrict__ kc, int kx, int ky, int L, int H, float4& a, float4& b)
{
    const bool up = ky >= H;
    const float4* r = kc + 2 * ((int64_t)kx * H + (up ? L - ky : ky));
    a = r[0];
    b = r[1];
    if (up) {
        b.z = -b.z;
        b.w = -b.w;
    }
}

// Kernel spectra, pass 1: rows a in [0, H) of the circulant embeddings of
// three packed complex kernels over node offsets (dx, dy), d^2 = s^2 |.|^2:
//   q = 0: K2 + i Ke/8      q = 1: K1 + i ln(eps + d^2)/1024
//   q = 2: K2 dx + i Ke dx / 8
// (rows a and L - a are equal, every kernel being even in dy), transformed
// along x; columns kx in [0, L/2] are kept (the kernels are even or odd in
// x), written column-major: krow[q][kx][a].
__device__ __forceinline__ void k_spec_rows_body(const GridDev* __restrict__ Gp, const float2* __restrict__ tw, float eps,
                            float2* __restrict__ krow, int sm_f2)
{
    extern __shared__ float2 smf[];
    __shared__ LinePlan pl;
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    const float s2 = G.s * G.s;
    make_line_plan(G, pl);
    const IpSmem sm = ip_smem(smf, sm_f2, L, true, true, tw);
    __syncthreads();
    make_digit_tables(pl, sm.drev, sm.pos_of);
    const int units = 3 * H;  // (q, a)
    int cap = sm.avail / L;
    cap = min(cap - !(cap & 1), (units + (int)gridDim.x - 1) / (int)gridDim.x);  // odd cap: ld = cap
    if (cap < 1) cap = 1;
    for (int u0 = blockIdx.x * cap; u0 < units; u0 += gridDim.x * cap) {
        const int nl = min(cap, units - u0), ld = nl | 1;
        const int nbp = (int)blockDim.x / nl, tl = (int)threadIdx.x % nl, tb = (int)threadIdx.x / nl;
        const int u = u0 + tl, q = u / H, a = u - q * H;
        __syncthreads();
        if (tb < nbp) {
            int dy;
            const bool rowok = circ_offset(a, M, L, dy);
            for (int b = tb; b < L; b += nbp) {
                int dx;
                float2 v = make_float2(0.f, 0.f);
                if (rowok && circ_offset(b, M, L, dx)) {
                    const float d2 = s2 * (float)(dx * dx + dy * dy);
                    const float k1 = 1.0f / (1.0f + d2);
                    const float ke = kEntScale / (eps + d2);
                    if (q == 0) v = make_float2(k1 * k1, ke);
                    else if (q == 1) v = make_float2(k1, kLnScale * logf(eps + d2));
                    else v = make_float2(k1 * k1 * (float)dx, ke * (float)dx);
                }
                sm.X[(int64_t)b * ld + tl] = v;
            }
        }
        __syncthreads();
        ip_fft<false>(sm.X, ld, nl, pl, sm.tw);
        if (tb < nbp)
            for (int kx = tb; kx < H; kx += nbp)
                krow[((int64_t)q * H + kx) * H + a] = sm.X[(int64_t)sm.pos_of[kx] * ld + tl];
    }
}

__global__ void __launch_bounds__(kIpThreads) k_spec_rows(const GridDev* __restrict__ Gp, const float2* __restrict__ tw, float eps,
                            float2* __restrict__ krow, int sm_f2)
{
    k_spec_rows_body(Gp, tw, eps, krow, sm_f2);
}

// Kernel spectra, pass 2: for tiles of columns kx, the three packed lines
// over a in [0, L) (mirrored from the H stored rows) transformed along y and
// unpacked into the records of kc_at, scaled by 1/L^2 (the inverse
// transforms are unnormalised):
//   FFT(K2 + i Ke/8) = K2^ + i Ke^/8,  FFT(K1 + i ln/1024) = K1^ + i ln^/1024,
//   FFT(K2 dx + i Ke dx/8) = i D2x + i (i Dex/8) = -Dex/8 + i D2x.
// Each column also supplies the transposed odd parts D?y of the records
// (ky, kx).
__device__ __forceinline__ void k_spec_cols_body(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                            const float2* __restrict__ krow, float4* __restrict__ kc, int sm_f2)
{
    extern __shared__ float2 smf[];
    __shared__ LinePlan pl;
    const GridDev& G = *Gp;
    const int L = G.L, H = L / 2 + 1;
    const float scale = 1.0f / ((float)L * (float)L);
    make_line_plan(G, pl);
    const IpSmem sm = ip_smem(smf, sm_f2, L, true, true, tw);
    __syncthreads();
    make_digit_tables(pl, sm.drev, sm.pos_of);
    int C = (sm.avail / L - 1) / 3;
    C = min(C, (H + (int)gridDim.x - 1) / (int)gridDim.x);
    if (C < 1) C = 1;
    for (int t = blockIdx.x; t * C < H; t += gridDim.x) {
        const int k0 = t * C, nc = min(C, H - k0), nl = 3 * nc;
        const int ld = (nl | 1) * L <= sm.avail ? (nl | 1) : nl;
        __syncthreads();
        // (line, a), a fastest: the mirrored rows, loads batched before the stores
        const int tot = nl * L;
        for (int i0 = threadIdx.x; i0 < tot; i0 += 8 * (int)blockDim.x) {
            float2 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * (int)blockDim.x;
                const int line = i / L, a = i - line * L;
                const int q = line / nc, c = line - q * nc;
                v[k] = i < tot ? krow[((int64_t)q * H + k0 + c) * H + (a < H ? a : L - a)] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * (int)blockDim.x;
                if (i < tot) {
                    const int line = i / L, a = i - line * L;
                    sm.X[(int64_t)a * ld + line] = v[k];
                }
            }
        }
        __syncthreads();
        ip_fft<false>(sm.X, ld, nl, pl, sm.tw);
        for (int c = 0; c < nc; ++c) {
            float4* rec = kc + 2 * ((int64_t)(k0 + c) * H);
            for (int ky = threadIdx.x; ky < H; ky += blockDim.x) {
                const float2* x = sm.X + (int64_t)sm.pos_of[ky] * ld + c;
                const float2 v0 = x[0], v1 = x[nc], v2 = x[2 * nc];
                rec[2 * ky] = make_float4(v0.x * scale, v0.y * scale / kEntScale, v1.x * scale, v1.y * scale / kLnScale);
                ((float2*)(rec + 2 * ky + 1))[0] = make_float2(v2.y * scale, -v2.x * scale / kEntScale);
            }
        }
        const int nbp = (int)blockDim.x / nc, tl = (int)threadIdx.x % nc, tb = (int)threadIdx.x / nc;
        if (tb < nbp)
            for (int ky = tb; ky < H; ky += nbp) {
                const float2 v2 = sm.X[(int64_t)sm.pos_of[ky] * ld + 2 * nc + tl];
                ((float2*)(kc + 2 * ((int64_t)ky * H + k0 + tl) + 1))[1] =
                    make_float2(v2.y * scale, -v2.x * scale / kEntScale);
            }
    }
}

__global__ void __launch_bounds__(kIpThreads) k_spec_cols(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                            const float2* __restrict__ krow, float4* __restrict__ kc, int sm_f2)
{
    k_spec_cols_body(Gp, tw, krow, kc, sm_f2);
}

// Row FFTs of the charge grids S0, S1x, S1y, S2 (node-local moments), packed
// two real rows per complex line (S0 + i S1x, S1y + i S2) and separated by
// Hermitian symmetry into half spectra srow[g][ty][kx], kx in [0, L/2].
// Tiles of T rows, line 2 r + pair, transformed in place (DIF); the
// Hermitian separation reads the digit-reversed positions of kx and L - kx.
__device__ __forceinline__ void k_conv_rows_fwd_body(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                                const float4* __restrict__ wflt, float2* __restrict__ srow, int sm_f2)
{
    extern __shared__ float2 smf[];
    __shared__ LinePlan pl;
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    make_line_plan(G, pl);
    const IpSmem sm = ip_smem(smf, sm_f2, L, true, true, tw);
    __syncthreads();
    make_digit_tables(pl, sm.drev, sm.pos_of);
    int T = (sm.avail / L - 1) / 2;
    T = min(T, (M + (int)gridDim.x - 1) / (int)gridDim.x);
    if (T < 1) T = 1;
    const int64_t MH = (int64_t)M * H;
    for (int t = blockIdx.x; t * T < M; t += gridDim.x) {
        const int r0 = t * T, nr = min(T, M - r0), nl = 2 * nr;
        const int ld = (nl | 1) * L <= sm.avail ? (nl | 1) : nl;
        __syncthreads();
        // (r, x) pairs, x fastest: one float4 of the charge grid feeds both
        // lines of row r; loads batched before the stores
        const int tot = nr * L;
        for (int i0 = threadIdx.x; i0 < tot; i0 += 8 * (int)blockDim.x) {
            float4 w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * (int)blockDim.x;
                const int r = i / L, x = i - r * L;
                w[k] = (i < tot && x < M) ? wflt[(int64_t)(r0 + r) * M + x] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * (int)blockDim.x;
                if (i < tot) {
                    const int r = i / L, x = i - r * L;
                    float2* dst = sm.X + (int64_t)x * ld + 2 * r;
                    dst[0] = make_float2(w[k].x, w[k].y);
                    dst[1] = make_float2(w[k].z, w[k].w);
                }
            }
        }
        __syncthreads();
        ip_fft<false>(sm.X, ld, nl, pl, sm.tw);
        for (int i = threadIdx.x; i < nl * H; i += blockDim.x) {
            const int l = i / H, k = i - l * H;
            const int r = l >> 1, pr = l & 1;
            const float2 z = sm.X[(int64_t)sm.pos_of[k] * ld + l];
            const float2 zc = conj2(sm.X[(int64_t)sm.pos_of[k == 0 ? 0 : L - k] * ld + l]);
            const float2 re = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y + zc.y));
            const float2 im = make_float2(0.5f * (z.y - zc.y), -0.5f * (z.x - zc.x));  // (z - zc) / 2i
            const int64_t o = (int64_t)(r0 + r) * H + k;
            srow[(int64_t)(2 * pr) * MH + o] = re;
            srow[(int64_t)(2 * pr + 1) * MH + o] = im;
        }
    }
}

__global__ void __launch_bounds__(kIpThreads) k_conv_rows_fwd(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                                const float4* __restrict__ wflt, float2* __restrict__ srow, int sm_f2)
{
    k_conv_rows_fwd_body(Gp, tw, wflt, srow, sm_f2);
}

// Column pass, tiles of columns kx in [0, L/2]: FFT along y of the four
// charge spectra (in place, digit-reversed out), the products with the kernel
// spectra (node-local form of the repulsion and entropy sums), inverse FFTs
// along y (conjugation trick, natural order out), rows < M kept:
//   U0 = K2^ S0^                 (F0)
//   U1 = Ke^ S0^                 (Fe0)
//   U2 = (K2 dx)^ S0^ - K2^ S1x^ (Vx)     U3 = (K2 dy)^ S0^ - K2^ S1y^ (Vy)
//   U4 = (Ke dx)^ S0^ - Ke^ S1x^ (Vex)    U5 = (Ke dy)^ S0^ - Ke^ S1y^ (Vey)
// and, by Parseval over the half spectrum, the grid sum
//   Z + n = sum [S0 (K1*S0) + 2 s^2 (S1 . (2 (K2 d)*S0 - K2*S1) + S2 (K2*S0))],
// accumulated in FP64 per column in an order fixed by the column alone
// (kColSlots warps, lanes over positions, a fixed tree), and finished by the
// last block in column order.
// Z integrand at (kx, ky) from the four charge spectra.
__device__ __forceinline__ float z_term(float2 s0, float2 s1x, float2 s1y, float2 s2v, float k2, float k1, float d2x,
                                        float d2y, float s2)
{
    const float gx_re = -2.0f * d2x * s0.y - k2 * s1x.x, gx_im = 2.0f * d2x * s0.x - k2 * s1x.y;
    const float gy_re = -2.0f * d2y * s0.y - k2 * s1y.x, gy_im = 2.0f * d2y * s0.x - k2 * s1y.y;
    const float t = k1 * (s0.x * s0.x + s0.y * s0.y);
    const float c = s1x.x * gx_re + s1x.y * gx_im + s1y.x * gy_re + s1y.y * gy_im + k2 * (s2v.x * s0.x + s2v.y * s0.y);
    return t + 2.0f * s2 * c;
}

// (K d)^ S0^ - K^ S1^ for an odd kernel spectrum i d (d real) and its even K.
__device__ __forceinline__ float2 odd_product(float d, float k, float2 s0, float2 s1)
{
    return make_float2(-d * s0.y - k * s1.x, d * s0.x - k * s1.y);
}

// Sum of one double per thread over the block (blockDim.x a multiple of 32,
// at most 1024): warp sums by shuffles, then warp 0 adds the warp sums in
// order (a fixed order, so the result is reproducible); every thread gets it.
__device__ __forceinline__ double block_sum_double(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}

constexpr int kColThreads = kIpThreads;
constexpr int kColSlots = 8;                        // warps per column in the Z sums
constexpr int kColMaxC = 16;                        // columns per tile

__device__ __forceinline__ void k_conv_cols_body(GridDev* Gp, const float2* __restrict__ tw, const float2* __restrict__ srow,
                            const float4* __restrict__ kc, float2* __restrict__ ucol, double* __restrict__ zcol,
                            int32_t n, int sm_f2)
{
    extern __shared__ float2 smf[];
    __shared__ LinePlan pl;
    __shared__ double wz[32], wl[32];
    __shared__ double red[33];
    __shared__ bool last;
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    const float s2 = G.s * G.s;
    make_line_plan(G, pl);
    // six lines per column; the twiddles move to global memory (L1) when
    // one column with them does not fit
    const bool tw_smem = 7 * L + L + (L + 3) / 4 <= sm_f2;
    const IpSmem sm = ip_smem(smf, sm_f2, L, false, tw_smem, tw);
    __syncthreads();
    make_digit_tables(pl, sm.drev, nullptr);
    int C = (sm.avail / L - 1) / 6;
    C = min(min(C, kColMaxC), (H + (int)gridDim.x - 1) / (int)gridDim.x);
    if (C < 1) C = 1;
    const int64_t MH = (int64_t)M * H;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nthr = (int)blockDim.x;                    // 256 or 512 threads
    const int per_round = (nthr >> 5) / kColSlots;       // columns per round of products
    for (int t = blockIdx.x; t * C < H; t += gridDim.x) {
        const int k0 = t * C, nc = min(C, H - k0);
        const int ld = (6 * nc + 1) * L <= sm.avail ? 6 * nc + 1 : 6 * nc;
        float2* X = sm.X;
        __syncthreads();
        {
            // line g nc + c: spectrum g of column k0 + c along y (rows >= M zero)
            const int nl = 4 * nc, nbp = nthr / nl, tl = (int)threadIdx.x % nl, tb = (int)threadIdx.x / nl;
            if (tb < nbp) {
                const int g = tl / nc, c = tl - g * nc;
                const float2* src = srow + g * MH + k0 + c;
                for (int y0 = tb; y0 < L; y0 += 8 * nbp) {
                    float2 v[8];  // loads issued before the stores
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int y = y0 + q * nbp;
                        v[q] = y < M ? src[(int64_t)y * H] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int y = y0 + q * nbp;
                        if (y < L) X[(int64_t)y * ld + tl] = v[q];
                    }
                }
            }
        }
        __syncthreads();
        ip_fft<false>(X, ld, 4 * nc, pl, sm.tw);
        // products in place at every position p (frequency drev[p]): line
        // q nc + c receives U_q of column k0 + c, conjugated for the inverse
        for (int c0 = 0; c0 < nc; c0 += per_round) {
            const int c = c0 + warp / kColSlots, wg = warp % kColSlots;
            double zp = 0.0, lp = 0.0;
            if (c < nc) {
                const int kx = k0 + c;
                const float wgt = (kx == 0 || 2 * kx == L) ? 1.0f : 2.0f;
                constexpr int kStride = 32 * kColSlots;
                for (int p0 = lane + 32 * wg; p0 < L; p0 += 4 * kStride) {
                    // the records of four positions fetched together
                    float4 ra[4], rb[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int p = p0 + q * kStride;
                        if (p < L) kc_at(kc, kx, sm.drev[p], L, H, ra[q], rb[q]);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                    const int p = p0 + q * kStride;
                    if (p >= L) break;
                    const float4 a = ra[q], b = rb[q];
                    float2* x = X + (int64_t)p * ld + c;
                    const float2 s0 = x[0], s1x = x[nc], s1y = x[2 * nc], s2v = x[3 * nc];
                    zp += (double)(wgt * z_term(s0, s1x, s1y, s2v, a.x, a.z, b.x, b.z, s2));
                    lp += (double)(wgt * a.w * (s0.x * s0.x + s0.y * s0.y));
                    x[0] = conj2(make_float2(a.x * s0.x, a.x * s0.y));
                    x[nc] = conj2(make_float2(a.y * s0.x, a.y * s0.y));
                    x[2 * nc] = conj2(odd_product(b.x, a.x, s0, s1x));
                    x[3 * nc] = conj2(odd_product(b.z, a.x, s0, s1y));
                    x[4 * nc] = conj2(odd_product(b.y, a.y, s0, s1x));
                    x[5 * nc] = conj2(odd_product(b.w, a.y, s0, s1y));
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                zp += __shfl_xor_sync(FULL, zp, o);
                lp += __shfl_xor_sync(FULL, lp, o);
            }
            if (lane == 0) {
                wz[warp] = zp;
                wl[warp] = lp;
            }
            __syncthreads();
            if ((int)threadIdx.x < per_round && c0 + (int)threadIdx.x < nc) {
                double zs = 0.0, ls = 0.0;
                for (int w = 0; w < kColSlots; ++w) {
                    zs += wz[threadIdx.x * kColSlots + w];
                    ls += wl[threadIdx.x * kColSlots + w];
                }
                zcol[k0 + c0 + threadIdx.x] = zs;
                zcol[H + k0 + c0 + threadIdx.x] = ls;
            }
            __syncthreads();
        }
        ip_fft<true>(X, ld, 6 * nc, pl, sm.tw);
        {
            const int nl = 6 * nc, nbp = nthr / nl, tl = (int)threadIdx.x % nl, tb = (int)threadIdx.x / nl;
            if (tb < nbp) {
                const int q = tl / nc, c = tl - q * nc;
                float2* dst = ucol + q * MH + k0 + c;
                for (int y = tb; y < M; y += nbp) dst[(int64_t)y * H] = conj2(X[(int64_t)y * ld + tl]);
            }
        }
    }
    // the last block to finish adds the column sums in column order (a
    // result that does not depend on how the columns were split over blocks)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&Gp->ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double v = 0.0, v2 = 0.0;
        for (int kx = threadIdx.x; kx < H; kx += blockDim.x) {
            v += ((volatile double*)zcol)[kx];
            v2 += ((volatile double*)zcol)[H + kx];
        }
        const double zt = block_sum_double(v, red);
        const double lt2 = block_sum_double(v2, red);
        if (threadIdx.x == 0) {
            Gp->Lsum = lt2;
            const double Z = zt - (double)n;
            Gp->Z = Z;
            Gp->SoZ = (float)(Gp->S / Z);
        }
    }
}

__global__ void __launch_bounds__(kColThreads) k_conv_cols(GridDev* Gp, const float2* __restrict__ tw, const float2* __restrict__ srow,
                            const float4* __restrict__ kc, float2* __restrict__ ucol, double* __restrict__ zcol,
                            int32_t n, int sm_f2)
{
    k_conv_cols_body(Gp, tw, srow, kc, ucol, zcol, n, sm_f2);
}

// Inverse row FFTs, three packed lines per row (U0 + i U1, U2 + i U3,
// U4 + i U5), each half spectrum extended by Hermitian symmetry.  Fields per
// node: f0 = F0, f1 = Vx, f2 = Vy, f3 = Fe0, f4 = Vex, f5 = Vey, f6 = f7 = 0.
// Tiles of T rows, line 3 r + pair, loaded straight into digit-reversed
// positions and transformed in place (DIT, conjugation trick), so each
// node's eight fields leave as one 32-byte record.  The plain (atomic)
// spread also needs the charge grid cleared for the next iteration; its
// readers have finished, so that is done here.
__device__ __forceinline__ void k_conv_rows_inv_body(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                                const float2* __restrict__ ucol, float* __restrict__ fields,
                                float4* __restrict__ wflt, int32_t* __restrict__ bcnt, int plain, int sm_f2)
{
    extern __shared__ float2 smf[];
    __shared__ LinePlan pl;
    const GridDev& G = *Gp;
    const int L = G.L, M = G.M, H = L / 2 + 1;
    make_line_plan(G, pl);
    const IpSmem sm = ip_smem(smf, sm_f2, L, true, true, tw);
    __syncthreads();
    make_digit_tables(pl, sm.drev, sm.pos_of);
    int T = (sm.avail / L - 1) / 3;
    T = min(T, (M + (int)gridDim.x - 1) / (int)gridDim.x);
    if (T < 1) T = 1;
    const int64_t MH = (int64_t)M * H;
    for (int t = blockIdx.x; t * T < M; t += gridDim.x) {
        const int r0 = t * T, nr = min(T, M - r0), nl = 3 * nr;
        const int ld = (nl | 1) * L <= sm.avail ? (nl | 1) : nl;
        __syncthreads();
        // (line, k) for k in [0, H), k fastest; k and L - k from one load pair
        const int tot = nl * H;
        for (int i0 = threadIdx.x; i0 < tot; i0 += 4 * (int)blockDim.x) {
            float2 a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * (int)blockDim.x;
                const int l = i / H, k = i - l * H;
                const int r = l / 3, pr = l - 3 * r;
                const float2* ua = ucol + (int64_t)(2 * pr) * MH + (int64_t)(r0 + r) * H + k;
                a[q] = i < tot ? ua[0] : make_float2(0.f, 0.f);
                b[q] = i < tot ? ua[MH] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * (int)blockDim.x;
                if (i < tot) {
                    const int l = i / H, k = i - l * H;
                    // conj(a + i b) at k; at L - k the half spectra are conjugated
                    sm.X[(int64_t)sm.pos_of[k] * ld + l] = conj2(make_float2(a[q].x - b[q].y, a[q].y + b[q].x));
                    if (k > 0 && 2 * k < L)
                        sm.X[(int64_t)sm.pos_of[L - k] * ld + l] =
                            conj2(make_float2(a[q].x + b[q].y, -a[q].y + b[q].x));
                }
            }
        }
        __syncthreads();
        ip_fft<true>(sm.X, ld, nl, pl, sm.tw);
        for (int i = threadIdx.x; i < nr * M; i += blockDim.x) {
            const int r = i / M, x = i - r * M;
            const float2* s = sm.X + (int64_t)x * ld + 3 * r;
            const float2 v0 = conj2(s[0]), v1 = conj2(s[1]), v2 = conj2(s[2]);
            float4* f = (float4*)(fields + ((int64_t)(r0 + r) * M + x) * kFieldStride);
            f[0] = make_float4(v0.x, v1.x, v1.y, v0.y);
            f[1] = make_float4(v2.x, v2.y, 0.f, 0.f);
        }
        if (plain)
            for (int i = threadIdx.x; i < nr * M; i += blockDim.x)
                wflt[(int64_t)r0 * M + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // the box counts of this iteration are used up: cleared for the next
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)G.I * G.I;
         t += (int64_t)gridDim.x * blockDim.x)
        bcnt[t] = 0;
}

__global__ void __launch_bounds__(kIpThreads) k_conv_rows_inv(const GridDev* __restrict__ Gp, const float2* __restrict__ tw,
                                const float2* __restrict__ ucol, float* __restrict__ fields,
                                float4* __restrict__ wflt, int32_t* __restrict__ bcnt, int plain, int sm_f2)
{
    k_conv_rows_inv_body(Gp, tw, ucol, fields, wflt, bcnt, plain, sm_f2);
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


// ---- batched wrappers: graph = blockIdx.y (BatchGraph), each graph's work
// split over gridDim.x blocks as in the single-graph launches ----
__device__ __forceinline__ const float2* layout_of(const BatchGraph& b, int parity) { return parity ? b.w.yalt : b.Y; }

__global__ void __launch_bounds__(kBoxThreads) k_setup_b(const BatchGraph* __restrict__ bg, int parity, float bwm,
                                                         int min_boxes, int P)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_setup_body(b.w.bounds + 2 * parity, b.w.bounds + 2 * (parity ^ 1), b.w.g, b.w.tw, layout_of(b, parity),
                 b.w.bcnt, b.n, bwm, min_boxes, b.max_boxes, P, 1);
}

__global__ void __launch_bounds__(kScanThreads) k_box_scan_b(const BatchGraph* __restrict__ bg)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_box_scan_body(b.w.g, b.w.bcnt, b.w.bcur, b.w.btot, b.w.bpre, b.w.heavy, b.w.items);
}

__global__ void __launch_bounds__(kBoxThreads) k_box_scatter_b(const BatchGraph* __restrict__ bg, int parity)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_box_scatter_body(layout_of(b, parity), b.n, b.w.g, b.w.bcur, b.w.bpre, b.w.su);
}

template <int P>
__global__ void __launch_bounds__(256) k_box_spread_b(const BatchGraph* __restrict__ bg)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_box_spread_body<P>(b.w.su, b.w.bcnt, b.w.bcur, b.w.bpre, b.w.heavy, b.w.items, b.w.hacc, b.w.hticket, b.w.g,
                         b.w.wflt);
}

__global__ void __launch_bounds__(kIpThreads) k_spec_rows_b(const BatchGraph* __restrict__ bg, float eps, int sm_f2)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_spec_rows_body(b.w.g, b.w.tw, eps, b.w.krow, sm_f2);
}

__global__ void __launch_bounds__(kIpThreads) k_spec_cols_b(const BatchGraph* __restrict__ bg, int sm_f2)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_spec_cols_body(b.w.g, b.w.tw, b.w.krow, b.w.kc, sm_f2);
}

__global__ void __launch_bounds__(kIpThreads) k_conv_rows_fwd_b(const BatchGraph* __restrict__ bg, int sm_f2)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_conv_rows_fwd_body(b.w.g, b.w.tw, b.w.wflt, b.w.srow, sm_f2);
}

__global__ void __launch_bounds__(kColThreads) k_conv_cols_b(const BatchGraph* __restrict__ bg, int sm_f2)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_conv_cols_body(b.w.g, b.w.tw, b.w.srow, b.w.kc, b.w.ucol, b.w.zcol, b.n, sm_f2);
}

__global__ void __launch_bounds__(kIpThreads) k_conv_rows_inv_b(const BatchGraph* __restrict__ bg, int sm_f2)
{
    const BatchGraph& b = bg[blockIdx.y];
    k_conv_rows_inv_body(b.w.g, b.w.tw, b.w.ucol, b.w.fields, b.w.wflt, b.w.bcnt, 0, sm_f2);
}
constexpr int kPsumBlocks = 304;

// Room for the twiddles plus six lines of the longest length (the column
// pass keeps four spectra and two work lines), at least 64 KB.
// Dynamic shared memory of every FFT pass: the most a block may take less a
// margin for the static arrays.  A fixed size makes every tiling decision a
// function of the grid alone.
constexpr size_t kFftSmemBytes = 230400;
// The batched FFT passes' half size: two blocks and their static shared
// memory per SM.
constexpr size_t kFftSmemHalf = 112640;
static_assert(kFftSmemBytes >= (size_t)(6 * kLMax + (kLMax + 3) / 4) * 8, "six FFT lines of kLMax must fit");

}  // namespace

IterShape iter_shape(int32_t n, const ltsnet_params* p)
{
    IterShape sh;
    sh.n = n;
    sh.P = p->nodes_per_box;
    sh.max_boxes = p->max_boxes;
    sh.Mmax = p->max_boxes * p->nodes_per_box;
    sh.Lmax = 2 * sh.Mmax;
    // boxes of more than kLightMax points: at most n / (kLightMax + 1)
    sh.hcap = std::min<int64_t>((int64_t)sh.max_boxes * sh.max_boxes, (int64_t)n / (kLightMax + 1) + 1);
    sh.conv_mode = p->conv_mode;
    return sh;
}

IterWs iter_carve(Carve& c, const IterShape& sh)
{
    IterWs w;
    const int64_t MM = (int64_t)sh.Mmax * sh.Mmax;
    w.st = c.take<StatusBlock>(1);
    w.g = c.take<GridDev>(1);
    w.bounds = c.take<int32_t>(4);
    w.tw = c.take<float2>(kLMax);
    const int64_t NB = (int64_t)sh.max_boxes * sh.max_boxes;
    w.bcnt = c.take<int32_t>(NB);
    w.bcur = c.take<int32_t>(NB);
    // boxes of more than kLightMax points: at most n / (kLightMax + 1) of
    // them, with at most n / kSeg + (their number) segments
    const int64_t HC = sh.hcap;
    w.heavy = c.take<int32_t>(HC);
    w.hticket = c.take<int32_t>(HC);
    w.hacc = c.take<long long>(HC * sh.P * sh.P * 4);
    w.items = c.take<int2>(HC + (int64_t)sh.n / kSeg + 1);
    w.btot = c.take<int32_t>(kMaxScanChunks);
    w.bpre = c.take<int32_t>(kMaxScanChunks);
    w.su = c.take<float2>(sh.n);
    w.wflt = c.take<float4>(MM);
    const int64_t HH = (int64_t)(sh.Lmax / 2 + 1) * (sh.Lmax / 2 + 1);
    const int64_t MH = (int64_t)sh.Mmax * (sh.Lmax / 2 + 1);
    w.krow = c.take<float2>(3 * HH);
    w.kc = c.take<float4>(2 * HH);
    w.srow = c.take<float2>(4 * MH);
    w.ucol = c.take<float2>(6 * MH);
    w.fields = c.take<float>(MM * kFieldStride);
    w.zblk = c.take<double>(1024);
    w.zcol = c.take<double>(2 * (sh.Lmax / 2 + 1));
    w.sblk = c.take<double>(1024);
    w.yalt = c.take<float2>(sh.n);
    w.phi = c.take<float>((int64_t)sh.n * 8);
    w.attr = c.take<float2>(sh.n);
    w.dft = DftWs{};
    if (sh.conv_mode == LTSNET_CONV_DFT_GEMM) dft_carve(c, sh, w.dft);
    return w;
}

// Clears what the iteration kernels expect cleared when a workspace is first
// used: the status block, the charge grid (the plain spread accumulates into
// it) and the heavy-box accumulators and tickets (cleared again by their
// last user every iteration).
cudaError_t iter_reset(const IterWs& w, const IterShape& sh, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.st, 0, sizeof(StatusBlock), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&w.g->imax, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.wflt, 0, sizeof(float4) * (size_t)sh.Mmax * sh.Mmax, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.hticket, 0, sizeof(int32_t) * (size_t)sh.hcap, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.bcnt, 0, sizeof(int32_t) * (size_t)sh.max_boxes * sh.max_boxes, s)) != cudaSuccess)
        return e;
    if (sh.conv_mode == LTSNET_CONV_DFT_GEMM && (e = dft_reset(w.dft, s)) != cudaSuccess) return e;
    return cudaMemsetAsync(w.hacc, 0, sizeof(long long) * (size_t)sh.hcap * sh.P * sh.P * 4, s);
}

cudaError_t launch_bounds_init(const IterWs& w, const float2* Y, int32_t n, int parity, cudaStream_t s)
{
    int32_t* b = w.bounds + 2 * parity;
    k_bounds_init<<<1, 1, 0, s>>>(b);
    int64_t blocks = ((int64_t)n + 255) / 256;
    if (blocks > num_sms() * 4) blocks = num_sms() * 4;
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
    int64_t sblocks = ((int64_t)n + kBoxTile - 1) / kBoxTile;
    if (sblocks > num_sms() * 4) sblocks = num_sms() * 4;
    if (sblocks < 16) sblocks = 16;
    k_setup<<<(unsigned)sblocks, kBoxThreads, 0, s>>>(w.bounds + 2 * parity, w.bounds + 2 * (parity ^ 1), w.g, w.tw,
                                                      Y, w.bcnt, n, p->box_width_max, p->min_boxes, p->max_boxes, P,
                                                      plain ? 0 : 1);
    count_launches(1);
    const size_t fsm = kFftSmemBytes;
    const int f2 = (int)(fsm / sizeof(float2));
    const int fb = num_sms();  // FFT blocks: one per SM
    // The kernel spectra need only the grid parameters: unless kernels are
    // being timed one by one, they run on a side stream next to the spread
    // and join before the column pass.
    AuxStreams* aux = nullptr;
    const bool fork = !profiling_active() && aux_streams(&aux) == cudaSuccess;
    if (fork) {
        cudaError_t e2;
        if ((e2 = cudaEventRecord(aux->fork, s)) != cudaSuccess) return e2;
        if ((e2 = cudaStreamWaitEvent(aux->branch, aux->fork, 0)) != cudaSuccess) return e2;
        k_spec_rows<<<fb, kIpThreads, fsm, aux->branch>>>(w.g, w.tw, p->eps, w.krow, f2);
        k_spec_cols<<<fb, kIpThreads, fsm, aux->branch>>>(w.g, w.tw, w.krow, w.kc, f2);
        count_launches(2);
        if ((e2 = cudaEventRecord(aux->join, aux->branch)) != cudaSuccess) return e2;
    }
    profile_start(LTSNET_KERNEL_SPREAD, s);
    if (plain) {
        int64_t blocks = ((int64_t)n + kBoxTile - 1) / kBoxTile;
        if (blocks > num_sms() * 8) blocks = num_sms() * 8;
        if (blocks < 1) blocks = 1;
        switch (P) {
            case 2: k_spread_atomic<2><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
            case 3: k_spread_atomic<3><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
            case 4: k_spread_atomic<4><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
            default: k_spread_atomic<5><<<(unsigned)blocks, 256, 0, s>>>(Y, n, w.g, w.wflt); break;
        }
        count_launches(1);
    } else {
        int64_t blocks = ((int64_t)n + kBoxTile - 1) / kBoxTile;
        if (blocks > num_sms() * 8) blocks = num_sms() * 8;
        if (blocks < 1) blocks = 1;
        const int nsb = std::min<int>(num_sms(), (int)(((int64_t)sh.max_boxes * sh.max_boxes + kScanBlock - 1) / kScanBlock));
        k_box_scan<<<nsb, kScanThreads, 0, s>>>(w.g, w.bcnt, w.bcur, w.btot, w.bpre, w.heavy, w.items);
        k_box_scatter<<<(unsigned)blocks, kBoxThreads, 0, s>>>(Y, n, w.g, w.bcur, w.bpre, w.su);
        switch (P) {
#define LT_SPREAD(PP)                                                                                      \
    case PP:                                                                                               \
        k_box_spread<PP><<<num_sms() * 4, 256, 0, s>>>(w.su, w.bcnt, w.bcur, w.bpre, w.heavy, w.items, w.hacc, \
                                                   w.hticket, w.g, w.wflt);                               \
        break;
            LT_SPREAD(2)
            LT_SPREAD(3)
            LT_SPREAD(4)
            default: LT_SPREAD(5)
#undef LT_SPREAD
        }
        count_launches(3);
    }
    profile_stop(LTSNET_KERNEL_SPREAD, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    profile_start(LTSNET_KERNEL_CONV, s);
    if (!fork) {
        k_spec_rows<<<fb, kIpThreads, fsm, s>>>(w.g, w.tw, p->eps, w.krow, f2);
        k_spec_cols<<<fb, kIpThreads, fsm, s>>>(w.g, w.tw, w.krow, w.kc, f2);
        count_launches(2);
    }
    if (sh.conv_mode == LTSNET_CONV_DFT_GEMM) {
        // DFT matrix products on the tensor cores (dftgemm.cu)
        if ((e = launch_dft_prep(w, s)) != cudaSuccess) return e;
        if (fork && (e = cudaStreamWaitEvent(s, aux->join, 0)) != cudaSuccess) return e;
        if ((e = launch_dft_products(w, n, s)) != cudaSuccess) return e;
        profile_stop(LTSNET_KERNEL_CONV, s);
        return cudaGetLastError();
    }
    k_conv_rows_fwd<<<fb, kIpThreads, fsm, s>>>(w.g, w.tw, w.wflt, w.srow, f2);
    if (fork) {
        cudaError_t e2 = cudaStreamWaitEvent(s, aux->join, 0);
        if (e2 != cudaSuccess) return e2;
    }
    k_conv_cols<<<fb, kColThreads, fsm, s>>>(w.g, w.tw, w.srow, w.kc, w.ucol, w.zcol, n, f2);
    k_conv_rows_inv<<<fb, kIpThreads, fsm, s>>>(w.g, w.tw, w.ucol, w.fields, w.wflt, w.bcnt, plain ? 1 : 0, f2);
    count_launches(3);
    profile_stop(LTSNET_KERNEL_CONV, s);
    return cudaGetLastError();
}

cudaError_t grid_set_smem_attrs()
{
    const int fsm = (int)kFftSmemBytes;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_spec_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_spec_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_spec_rows_b, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_spec_cols_b, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_rows_fwd_b, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_cols_b, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    if ((e = cudaFuncSetAttribute(k_conv_rows_inv_b, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm))) return e;
    return cudaSuccess;
}

// The grid phase of one iteration for every graph of a batch: the same
// kernels and order as launch_grid_phase, each launch covering all graphs
// (grid.y = graph).  sh is the shape of the batch's largest grid (shared
// memory of the FFT passes); point-indexed kernels get enough blocks per
// graph for the largest graph and the others leave theirs idle.
cudaError_t launch_grid_phase_batched(const BatchGraph* bg, int32_t ng, const BatchShape& bs, const IterShape& sh,
                                      const ltsnet_params* p, int parity, cudaStream_t s)
{
    const int P = sh.P;
    const unsigned tiles = (unsigned)std::max<int64_t>(1, ((int64_t)bs.max_n + kBoxTile - 1) / kBoxTile);
    const dim3 gpt(tiles, (unsigned)ng);
    k_setup_b<<<gpt, kBoxThreads, 0, s>>>(bg, parity, p->box_width_max, p->min_boxes, P);
    count_launches(1);
    // FFT blocks sized for the batch's largest grid cap: when half the
    // shared memory holds one column of it (seven lines and the digit
    // table), blocks of 256 threads and half the shared memory run two to
    // an SM; every line is transformed the same way whatever the block, so
    // each graph's result does not change.
    size_t fsm = kFftSmemBytes;
    unsigned fthr = kIpThreads;
    if ((size_t)(15 * sh.Lmax / 2 + 64) * sizeof(float2) <= kFftSmemHalf) {
        fsm = kFftSmemHalf;
        fthr = kIpThreads / 2;
    }
    const int f2 = (int)(fsm / sizeof(float2));
    const dim3 gfft((unsigned)bs.fft_blocks, (unsigned)ng);
    AuxStreams* aux = nullptr;
    const bool fork = !profiling_active() && aux_streams(&aux) == cudaSuccess;
    cudaError_t e;
    if (fork) {
        if ((e = cudaEventRecord(aux->fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(aux->branch, aux->fork, 0)) != cudaSuccess) return e;
        k_spec_rows_b<<<gfft, fthr, fsm, aux->branch>>>(bg, p->eps, f2);
        k_spec_cols_b<<<gfft, fthr, fsm, aux->branch>>>(bg, f2);
        count_launches(2);
        if ((e = cudaEventRecord(aux->join, aux->branch)) != cudaSuccess) return e;
    }
    const int64_t nb = (int64_t)sh.max_boxes * sh.max_boxes;
    const unsigned nsb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4, (nb + kScanBlock - 1) / kScanBlock));
    k_box_scan_b<<<dim3(nsb, (unsigned)ng), kScanThreads, 0, s>>>(bg);
    k_box_scatter_b<<<gpt, kBoxThreads, 0, s>>>(bg, parity);
    const dim3 gsp((unsigned)bs.spread_blocks, (unsigned)ng);
    switch (P) {
        case 2: k_box_spread_b<2><<<gsp, 256, 0, s>>>(bg); break;
        case 3: k_box_spread_b<3><<<gsp, 256, 0, s>>>(bg); break;
        case 4: k_box_spread_b<4><<<gsp, 256, 0, s>>>(bg); break;
        default: k_box_spread_b<5><<<gsp, 256, 0, s>>>(bg); break;
    }
    count_launches(3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!fork) {
        k_spec_rows_b<<<gfft, fthr, fsm, s>>>(bg, p->eps, f2);
        k_spec_cols_b<<<gfft, fthr, fsm, s>>>(bg, f2);
        count_launches(2);
    }
    k_conv_rows_fwd_b<<<gfft, fthr, fsm, s>>>(bg, f2);
    if (fork && (e = cudaStreamWaitEvent(s, aux->join, 0)) != cudaSuccess) return e;
    k_conv_cols_b<<<gfft, fthr, fsm, s>>>(bg, f2);
    k_conv_rows_inv_b<<<gfft, fthr, fsm, s>>>(bg, f2);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace lt
