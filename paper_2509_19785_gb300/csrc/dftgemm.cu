// Grid convolution of the interpolation (Sec. 2.3 "four sums", Sec. 3.3
// entropy sums, Alg. 3 loop) as dense DFT matrix products on the tensor cores:
// conv_mode 1, the alternative to the FFT of grid.cu.
//
// Both forms compute the same node-local sums (grid.cu's header): the charge
// grids S0, S1x, S1y, S2 (M x M) are convolved, zero padded to L = 2M, with
// the kernels (1+d^2)^-2 and 1/(eps+d^2) and with those kernels times the
// node offset, and Z and the entropy double sum come from the same spectra
// by Parseval.  Here every transform is a real matrix product.  With
// c(t,k) = cos(2 pi t k / L), s(t,k) = sin(2 pi t k / L) and k in [0, H),
// H = L/2 + 1, a charge grid W has the four real spectra
//   T^{ab}[ky,kx] = sum_{y,x} W[y,x] a(y,ky) b(x,kx),   a, b in {c, s}.
// A kernel even in dx and dy has a real spectrum K^ (even in ky and kx), and
// K*W = sum_{ab} Inv_ab(K^ T^{ab}) with Inv_ab(Q)[y,x] = sum_k w_ky w_kx
// a(y,ky) b(x,kx) Q[ky,kx] / L^2 (w = 1 at k = 0 and L/2, else 2: the two
// halves of the spectrum folded onto one).  A kernel odd in dx has the
// spectrum -i D (D real, odd in kx) and contributes sigma(b) D T^{a bbar} to
// the (a, b) inverse (sigma(s) = +1, sigma(c) = -1, bbar the other of c, s);
// odd in dy likewise with sigma(a) and abar.  The five products:
//   S1  T1[(kx,b), (g,y)] = sum_x F[(kx,b), x] W_g[y,x]        x-transforms
//   S2  T [(kx,g,b), (ky,a)] = sum_y T1 F[(ky,a), y]            y-transforms
//   (k_dft_products) per (ky, kx) the kernel products Q_q^{ab} of the six
//       fields and the Parseval sums of Z and of the entropy double sum
//   S4  R[y', (q,kx,b)] = sum_{(ky,a)} F[(ky,a), y'] Q          inverse in y
//   S5  f_q[y', x'] = sum_{(kx,b)} R F[(kx,b), x']              inverse in x
// F[(k,a), t] = a(t, k) is one table (stored twice, once per operand shape).
//
// Precision: every FP32 operand is split into three BF16 terms
// v0 = bf16(v), v1 = bf16(v - v0), v2 = bf16(v - v0 - v1), which hold its 24
// significand bits, and each product is the six tensor-core products
// a_i b_j with i + j <= 2, accumulated in FP32 in tensor memory (the three
// dropped products are below 2^-24 of the result).  Two terms with three
// products (16 bits per operand) left the fields about 1e-5 off.
//
// Layout of an operand matrix (rows x K, BF16, one plane per split term):
// blocks of 128 rows x 64 K elements (16 KB) in row-block-major order; inside
// a block, core matrices of 8 rows x 8 K elements (128 bytes, rows 16 bytes
// apart), core (m, k) at (8 m + k) * 128 bytes.  A 128 x 64 operand tile is
// one contiguous 16 KB copy (cp.async.bulk) and is described to tcgen05.mma
// as a K-major, unswizzled matrix with 128 bytes between K-adjacent and 1024
// bytes between row-adjacent core matrices.  Epilogues write the next
// product's operand directly in this layout, 8 K elements (16 bytes) at a
// time.
//
// Every operand's padding (rows and K beyond the valid extent) is rewritten
// with zeros in every iteration by the kernel that writes the operand, so a
// grid that shrinks leaves nothing stale behind.
#include <cuda_bf16.h>

#include <algorithm>

#include "iter.cuh"
#include "tc.cuh"

namespace lt {

namespace {

constexpr int kGemmThreads = 256;  // warp 0 loads, warp 1 issues MMAs, warp 2 owns TMEM, warps 4-7 epilogue
constexpr int kTerms = 3;          // BF16 terms per operand
constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr uint32_t kBlockElems = kBM * kBK;     // 8192 BF16 = 16 KB
constexpr uint32_t kBlockBytes = kBlockElems * 2;

__host__ __device__ constexpr int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

struct DftDims {
    int M, L, H, Mp, Kf;  // nodes per dim, FFT length, spectrum half length, M and 2H padded to 64
};

__device__ __forceinline__ DftDims dft_dims(const GridDev* G)
{
    DftDims d;
    d.M = G->M;
    d.L = G->L;
    d.H = d.L / 2 + 1;
    d.Mp = (int)rup(d.M, 64);
    d.Kf = (int)rup(2 * d.H, 64);
    return d;
}

// Element offset of (r, k) in an operand matrix with nkb K blocks.
__device__ __forceinline__ int64_t kt_off(int64_t r, int k, int nkb)
{
    return ((r >> 7) * nkb + (k >> 6)) * (int64_t)kBlockElems + ((((r >> 3) & 15) << 3) + ((k >> 3) & 7)) * 64 +
           (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// Eight consecutive K elements split into their BF16 terms and stored at
// element offset `off` of each plane (16-byte stores; planes `plane`
// elements apart).  Each residual is exact in FP32.
__device__ __forceinline__ void store_split8(uint16_t* base, int64_t plane, int64_t off, const float* f)
{
    float r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = f[i];
#pragma unroll
    for (int t = 0; t < kTerms; ++t) {
        float h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            h[i] = __bfloat162float(__float2bfloat16_rn(r[i]));
            r[i] -= h[i];
        }
        *(uint4*)(base + t * plane + off) = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]),
                                                       pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
    }
}

__device__ __forceinline__ void store_zero8(uint16_t* base, int64_t plane, int64_t off)
{
#pragma unroll
    for (int t = 0; t < kTerms; ++t) *(uint4*)(base + t * plane + off) = make_uint4(0u, 0u, 0u, 0u);
}

// a(t, k) from the twiddles tw[u] = e^{-2 pi i u / L}: cos for a = 0, sin for 1.
__device__ __forceinline__ float trig(const float2* __restrict__ tw, int t, int k, int a, int L)
{
    const float2 e = tw[(int)(((int64_t)t * k) % L)];
    return a ? -e.y : e.x;
}

// Tables, rebuilt only when the grid size changed (the S1 product records
// the size it was built for): F (rows (k, a) = 2k + a, K = node t) and its
// transpose G (rows t, K = 2k + a), zero outside k < H, t < M, written over
// their whole padded extents.
__global__ void k_dft_tables(const GridDev* __restrict__ G, const float2* __restrict__ tw, DftWs w)
{
    const DftDims d = dft_dims(G);
    if (*(volatile int32_t*)w.tabM == d.M) return;
    const int nF = d.Mp / 8, nG = d.Kf / 8;  // 8-element chunks per row
    const int64_t rowsF = rup(d.Kf, 256), rowsG = rup(d.Mp, 256);
    const int64_t totF = rowsF * nF, tot = totF + rowsG * nG;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < tot; u += (int64_t)gridDim.x * blockDim.x) {
        float v[8];
        if (u < totF) {
            const int64_t r = u / nF;
            const int k0 = (int)(u - r * nF) * 8;
            const int kk = (int)(r >> 1), a = (int)(r & 1);
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = (kk < d.H && k0 + i < d.M) ? trig(tw, k0 + i, kk, a, d.L) : 0.f;
            store_split8(w.F, w.pF, kt_off(r, k0, d.Mp / kBK), v);
        } else {
            const int64_t uu = u - totF;
            const int64_t r = uu / nG;
            const int k0 = (int)(uu - r * nG) * 8;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int kk = (k0 + i) >> 1, a = (k0 + i) & 1;
                v[i] = (kk < d.H && r < d.M) ? trig(tw, (int)r, kk, a, d.L) : 0.f;
            }
            store_split8(w.G, w.pG, kt_off(r, k0, d.Kf / kBK), v);
        }
    }
}

// The charge grids as the S1 operand: rows g * Mp + y, K = x, zero padded;
// also clears the box counts for the next iteration (their last reader, the
// spread, has finished).
__global__ void k_dft_charges(const GridDev* __restrict__ G, const float4* __restrict__ wflt, DftWs w,
                              int32_t* __restrict__ bcnt)
{
    const DftDims d = dft_dims(G);
    const int nc = d.Mp / 8;
    const int64_t tot = (int64_t)4 * d.Mp * nc;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = tid; u < tot; u += nth) {
        const int64_t r = u / nc;
        const int x0 = (int)(u - r * nc) * 8;
        const int g = (int)(r / d.Mp), y = (int)(r - (int64_t)g * d.Mp);
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float c = 0.f;
            if (y < d.M && x0 + i < d.M) {
                const float4 q = wflt[(int64_t)y * d.M + x0 + i];
                c = g == 0 ? q.x : (g == 1 ? q.y : (g == 2 ? q.z : q.w));
            }
            v[i] = c;
        }
        store_split8(w.W, w.pW, kt_off(r, x0, d.Mp / kBK), v);
    }
    const int64_t nb = (int64_t)G->I * G->I;
    for (int64_t t = tid; t < nb; t += nth) bcnt[t] = 0;
}


struct GemmArgs {
    GridDev* G;
    StatusBlock* st;
    DftWs w;
    float* fields;      // M x M nodes x 8 fields
    double* zblk;       // per-block partial sums of Z (first 512) and of the entropy sum (next 512)
    int32_t n;
};

// Operands, tile grid and K blocks of product ST at the current dimensions.
struct StageGeo {
    const uint16_t *A, *B;
    int64_t pA, pB;  // plane strides
    int Rm, Cn, nkb;
};

template <int ST, int BN>
__device__ __forceinline__ StageGeo stage_geo(const DftDims& d, const DftWs& w)
{
    StageGeo g;
    if (ST == 1) {
        g.A = w.F; g.pA = w.pF; g.B = w.W; g.pB = w.pW;
        g.Rm = (int)rup(d.Kf, kBM); g.Cn = 4 * d.Mp; g.nkb = d.Mp / kBK;
    } else if (ST == 2) {
        g.A = w.X; g.pA = w.pX; g.B = w.F; g.pB = w.pF;
        g.Rm = 4 * d.Kf; g.Cn = (int)rup(d.Kf, BN); g.nkb = d.Mp / kBK;
    } else if (ST == 3) {
        g.A = w.G; g.pA = w.pG; g.B = w.Q; g.pB = w.pQ;
        g.Rm = (int)rup(d.Mp, kBM); g.Cn = (int)rup(6 * d.Kf, BN); g.nkb = d.Kf / kBK;
    } else {
        g.A = w.R; g.pA = w.pR; g.B = w.G; g.pB = w.pG;
        g.Rm = 8 * d.Mp; g.Cn = (int)rup(d.M, BN); g.nkb = d.Kf / kBK;
    }
    return g;
}

// ---- epilogues: one thread holds row `row` of the product tile, columns
// c0 .. c0+31 in v ----

// S1: rows (kx, b) = 2 kx + b of the x-transforms, columns g * Mp + y; writes
// the S2 operand rows 8 kx + 2 g + b, K = y.
__device__ __forceinline__ void epi_s1(const GemmArgs& a, const DftDims& d, int row, int c0, const float* v)
{
    if (row >= d.Kf) return;
    const int kx = row >> 1, b = row & 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = c0 + 8 * j;
        const int g = col / d.Mp, y0 = col - g * d.Mp;
        store_split8(a.w.X, a.w.pX, kt_off((int64_t)kx * 8 + g * 2 + b, y0, d.Mp / kBK), v + 8 * j);
    }
}

__device__ __forceinline__ float fold_w(int k, int H) { return (k == 0 || k == H - 1) ? 1.0f : 2.0f; }

// S2: rows 8 kx + 2 g + b, columns 2 ky + a: the four charges' spectra
// T_g^{ab}[ky, kx], written in FP32 (rows of Kf floats) for k_dft_products.
__device__ __forceinline__ void epi_s2(const GemmArgs& a, const DftDims& d, int row, int c0, const float* v)
{
    if (c0 >= d.Kf) return;
    float4* t = (float4*)(a.w.T + (int64_t)row * d.Kf + c0);
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// S4: rows y' (inverse in y), columns q Kf + 2 kx + b; writes the S5 operand
// rows 8 y' + q, K = 2 kx + b (slots 6 and 7 zero).
__device__ __forceinline__ void epi_s4(const GemmArgs& a, const DftDims& d, int row, int c0, const float* v)
{
    if (row >= d.Mp) return;
    const int nkb = d.Kf / kBK;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = c0 + 8 * j;
        const int q = col / d.Kf, k0 = col - q * d.Kf;
        if (q >= 6) break;
        store_split8(a.w.R, a.w.pR, kt_off((int64_t)row * 8 + q, k0, nkb), v + 8 * j);
        if (q == 5) {
            store_zero8(a.w.R, a.w.pR, kt_off((int64_t)row * 8 + 6, k0, nkb));
            store_zero8(a.w.R, a.w.pR, kt_off((int64_t)row * 8 + 7, k0, nkb));
        }
    }
}

// S5: rows 8 y' + q, columns x'; field slot q of node (y', x').
__device__ __forceinline__ void epi_s5(const GemmArgs& a, const DftDims& d, int row, int c0, const float* v)
{
    const int y = row >> 3, q = row & 7;
    if (y >= d.M) return;
    float* f = a.fields + ((int64_t)y * d.M) * kFieldStride + q;
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if (c0 + i < d.M) f[(int64_t)(c0 + i) * kFieldStride] = v[i];
}

template <int BN>
constexpr size_t gemm_smem_bytes()
{
    return 2 * (kTerms * (size_t)kBlockBytes + kTerms * (size_t)BN * kBK * 2) + 1024 + 256;
}

// One product of the DFT chain: D = A B^T with A, B in split-BF16 operand
// layout, persistent over the tiles (BM = 128 rows x BN columns), two-stage
// operand pipeline and two TMEM accumulators (the epilogue of one tile runs
// while the next tile's products are issued).
template <int ST, int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) k_dft_gemm(GemmArgs a)
{
    extern __shared__ unsigned char smraw[];
    constexpr uint32_t kBTile = (uint32_t)BN * kBK * 2;  // one split term of a B tile
    constexpr uint32_t kStage = kTerms * (kBlockBytes + kBTile);  // A terms, then B terms
    constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kBM, BN);
    unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t* bar = (uint64_t*)(sm + 2 * kStage);  // full[2], empty[2], tfull[2], tempty[2], fin
    uint64_t* full = bar;
    uint64_t* empty = bar + 2;
    uint64_t* tfull = bar + 4;
    uint64_t* tempty = bar + 6;
    uint64_t* fin = bar + 8;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const DftDims d = dft_dims(a.G);
    const StageGeo geo = stage_geo<ST, BN>(d, a.w);
    const int nmt = geo.Rm / kBM, nnt = geo.Cn / BN;
    const int ntiles = nmt * nnt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (ST == 1 && blockIdx.x == 0 && threadIdx.x == 0) *a.w.tabM = d.M;  // tables are built for this size
    const bool work = (int)blockIdx.x < ntiles;

    if (work) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < 2; ++i) {
                tc::mbar_init(&full[i], 1);
                tc::mbar_init(&empty[i], 1);
                tc::mbar_init(&tfull[i], 1);
                tc::mbar_init(&tempty[i], 4);
            }
            tc::mbar_init(fin, 1);
            tc::mbar_fence_init();
            abort_flag = 0;
        }
        if (warp == 2) {
            tc::tmem_alloc(&tmem_slot, 2 * BN);
            tc::tmem_relinquish();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        const uint32_t tmem = tmem_slot;
        volatile int* abort = &abort_flag;

        if (warp == 0 && lane == 0) {
            // producer: bulk copies of the A and B tiles, two stages
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int mt = t % nmt, nt = t / nmt;
                for (int kb = 0; kb < geo.nkb; ++kb, ++it) {
                    const int s = it & 1;
                    const uint32_t ph = (it >> 1) & 1;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1, abort)) { ok = false; break; }
                    unsigned char* sa = sm + s * kStage;
                    tc::mbar_arrive_expect_tx(&full[s], kStage);
                    const int64_t ao = ((int64_t)mt * geo.nkb + kb) * kBlockElems;
#pragma unroll
                    for (int q = 0; q < kTerms; ++q) {
                        tc::bulk_g2s(sa + q * kBlockBytes, geo.A + q * geo.pA + ao, kBlockBytes, &full[s]);
#pragma unroll
                        for (int j = 0; j < BN / kBM; ++j) {
                            const int64_t bo = ((int64_t)(nt * (BN / kBM) + j) * geo.nkb + kb) * kBlockElems;
                            tc::bulk_g2s(sa + kTerms * kBlockBytes + q * kBTile + j * kBlockBytes,
                                         geo.B + q * geo.pB + bo, kBlockBytes, &full[s]);
                        }
                    }
                }
            }
            if (!ok) {
                record_error(a.st, LTSNET_ERR_DEVICE_TIMEOUT, 0x100 * ST + 1);
                *abort = 1;
            }
            // copies still in flight land before the block exits
            for (uint32_t k = (it > 2 ? it - 2 : 0); k < it; ++k)
                tc::mbar_wait(&full[k & 1], (k >> 1) & 1, nullptr);
        } else if (warp == 1 && lane == 0) {
            // MMA issuer: six split-term products per K step of 16.  Each K
            // block (64) goes into its own accumulator (unit u in TMEM buffer
            // u % 2); the epilogue adds the blocks in FP32 registers, so the
            // tensor core never accumulates more than one block.
            bool ok = true;
            uint32_t it = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int kb = 0; kb < geo.nkb; ++kb, ++it) {
                    const int acc = it & 1;
                    if (!tc::mbar_wait(&tempty[acc], ((it >> 1) & 1) ^ 1, abort)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t dt = tmem + (uint32_t)(acc * BN);
                    const int s = it & 1;
                    if (!tc::mbar_wait(&full[s], (it >> 1) & 1, abort)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_addr(sm + s * kStage);
                    const uint32_t sb = sa + kTerms * kBlockBytes;
#pragma unroll
                    for (int j = 0; j < kBK / 16; ++j) {
                        uint64_t ad[kTerms], bd[kTerms];
#pragma unroll
                        for (int q = 0; q < kTerms; ++q) {
                            ad[q] = tc::smem_desc(sa + q * kBlockBytes + j * 256, 128, 1024);
                            bd[q] = tc::smem_desc(sb + q * kBTile + j * 256, 128, 1024);
                        }
                        // a_i b_j for i + j <= 2, largest terms first
                        tc::mma_bf16(dt, ad[0], bd[0], kIdesc, j != 0);
                        tc::mma_bf16(dt, ad[0], bd[1], kIdesc, 1u);
                        tc::mma_bf16(dt, ad[1], bd[0], kIdesc, 1u);
                        tc::mma_bf16(dt, ad[0], bd[2], kIdesc, 1u);
                        tc::mma_bf16(dt, ad[1], bd[1], kIdesc, 1u);
                        tc::mma_bf16(dt, ad[2], bd[0], kIdesc, 1u);
                    }
                    tc::mma_commit(&empty[s]);
                    tc::mma_commit(&tfull[acc]);
                }
            }
            if (!ok) {
                record_error(a.st, LTSNET_ERR_DEVICE_TIMEOUT, 0x100 * ST + 2);
                *abort = 1;
            }
            // every product issued here has completed before TMEM is released
            tc::mma_commit(fin);
            tc::mbar_wait(fin, 0, nullptr);
        } else if (warp >= 4) {
            // epilogue: TMEM lane quarter (warp % 4), one tile row per thread;
            // the K blocks of a tile are summed here in FP32, then the tile's
            // row goes through the product's epilogue
            const int eq = warp - 4;
            const uint32_t lane_base = tmem + ((uint32_t)(eq * 32) << 16);
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int mt = t % nmt, nt = t / nmt;
                float acc[BN];
                for (int kb = 0; kb < geo.nkb; ++kb, ++it) {
                    const int ab = it & 1;
                    if (!tc::mbar_wait(&tfull[ab], (it >> 1) & 1, abort)) {
                        if (lane == 0) record_error(a.st, LTSNET_ERR_DEVICE_TIMEOUT, 0x100 * ST + 3);
                        *abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
#pragma unroll
                    for (int c = 0; c < BN / 32; ++c) {
                        float v[32];
                        tc::tmem_ld32(lane_base + (uint32_t)(ab * BN + c * 32), v);
#pragma unroll
                        for (int i = 0; i < 32; ++i) acc[c * 32 + i] = kb == 0 ? v[i] : acc[c * 32 + i] + v[i];
                    }
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tempty[ab]);
                }
                if (!ok) break;
                const int row = mt * kBM + eq * 32 + lane;
#pragma unroll
                for (int c = 0; c < BN / 32; ++c) {
                    const int c0 = nt * BN + c * 32;
                    if (ST == 1) epi_s1(a, d, row, c0, acc + c * 32);
                    else if (ST == 2) epi_s2(a, d, row, c0, acc + c * 32);
                    else if (ST == 3) epi_s4(a, d, row, c0, acc + c * 32);
                    else epi_s5(a, d, row, c0, acc + c * 32);
                }
            }
        }
        __syncthreads();
        if (warp == 2) {
            tc::fence_after_sync();
            tc::tmem_dealloc(tmem, 2 * BN);
        }
    }
}

// The kernel products between S2 and S4, and the Parseval sums.  Thread
// unit (kx, 4 consecutive ky): reads the four charges' spectra T_g^{ab}
// (rows 8 kx + 2 g + b of T, columns 2 ky + a) and the packed kernel values,
// forms for each b the six fields' products Q_q^{ab} (slot order F0, Vx, Vy,
// Fe0, Vex, Vey; slots 6, 7 zero) as the S4 operand rows q Kf + 2 kx + b,
// K = 2 ky + a, and adds the Z + n and entropy double-sum terms:
//   Z + n = sum_k sum_ab [K1 T0 T0 + 2 s^2 (T1 (2 sigma(b) D2x T0^{a bbar}
//           - K2 T1) + T2 (2 sigma(a) D2y T0^{abar b} - K2 T2) + K2 T3 T0)]
//   sum ln = sum_k sum_ab Kln T0 T0.
// Units with kx or ky >= H write zeros (padding of the S4 operand).  Each
// thread sums in FP64 in a fixed order, the block in a fixed order, and the
// last block adds the block sums in block order.
constexpr int kProdThreads = 256;

__global__ void __launch_bounds__(kProdThreads) k_dft_products(GridDev* G, DftWs w, const float4* __restrict__ kp,
                                                                StatusBlock* st, double* __restrict__ zblk, int32_t n)
{
    __shared__ double red[2][kProdThreads / 32];
    __shared__ bool last;
    const DftDims d = dft_dims(G);
    const int H = d.H, Kf = d.Kf, nkb = Kf / kBK;
    const float s2 = G->s * G->s;
    const int nky4 = Kf / 8, nkx = Kf / 2;
    const int64_t units = (int64_t)nkx * nky4;
    double zacc = 0.0, lacc = 0.0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(u / nky4), ky0 = (int)(u - (int64_t)kx * nky4) * 4;
        // T[g][b][a] for the 4 ky of the unit
        float Tv[4][2][4][2];
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float4* src = (const float4*)(w.T + (int64_t)(8 * kx + 2 * g + b) * Kf + 2 * ky0);
                const float4 p = src[0], q = src[1];
                Tv[g][b][0][0] = p.x; Tv[g][b][0][1] = p.y; Tv[g][b][1][0] = p.z; Tv[g][b][1][1] = p.w;
                Tv[g][b][2][0] = q.x; Tv[g][b][2][1] = q.y; Tv[g][b][3][0] = q.z; Tv[g][b][3][1] = q.w;
            }
        float Q[8][2][8];  // [q][b][2 ky' + a]
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int ky = ky0 + i;
            float4 ka = make_float4(0.f, 0.f, 0.f, 0.f), kb = ka;
            if (kx < H && ky < H) {
                const int64_t o = ((int64_t)kx * H + ky) * 2;
                ka = kp[o];
                kb = kp[o + 1];
            }
            const float k2 = ka.x, ke = ka.y, k1 = ka.z, kl = ka.w;
            const float d2x = kb.x, dex = kb.y, d2y = kb.z, dey = kb.w;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float sb = b ? 1.0f : -1.0f;
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float sa = a ? 1.0f : -1.0f;
                    const float o0 = Tv[0][b][i][a], x0 = Tv[0][b ^ 1][i][a], o0b = Tv[0][b][i][a ^ 1];
                    const float t1 = Tv[1][b][i][a], t2 = Tv[2][b][i][a], t3 = Tv[3][b][i][a];
                    Q[0][b][2 * i + a] = k2 * o0;
                    Q[1][b][2 * i + a] = sb * d2x * x0 - k2 * t1;
                    Q[2][b][2 * i + a] = sa * d2y * o0b - k2 * t2;
                    Q[3][b][2 * i + a] = ke * o0;
                    Q[4][b][2 * i + a] = sb * dex * x0 - ke * t1;
                    Q[5][b][2 * i + a] = sa * dey * o0b - ke * t2;
                    Q[6][b][2 * i + a] = 0.f;
                    Q[7][b][2 * i + a] = 0.f;
                    const float z = k1 * o0 * o0 + 2.0f * s2 * (t1 * (2.0f * sb * d2x * x0 - k2 * t1) +
                                                                t2 * (2.0f * sa * d2y * o0b - k2 * t2) + k2 * t3 * o0);
                    zacc += (double)z;
                    lacc += (double)(kl * o0 * o0);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int b = 0; b < 2; ++b)
                store_split8(w.Q, w.pQ, kt_off((int64_t)q * Kf + 2 * kx + b, 2 * ky0, nkb), Q[q][b]);
    }
    // fixed-order reductions: warp, block, then blocks in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zacc += __shfl_xor_sync(FULL, zacc, o);
        lacc += __shfl_xor_sync(FULL, lacc, o);
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][wid] = zacc;
        red[1][wid] = lacc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double zs = 0.0, ls = 0.0;
        for (int i = 0; i < kProdThreads / 32; ++i) {
            zs += red[0][i];
            ls += red[1][i];
        }
        zblk[blockIdx.x] = zs;
        zblk[512 + blockIdx.x] = ls;
        __threadfence();
        last = atomicAdd(&G->ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double zt = 0.0, lt2 = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            zt += ((volatile double*)zblk)[b];
            lt2 += ((volatile double*)zblk)[512 + b];
        }
        const double Z = zt - (double)n;
        G->Z = Z;
        G->Lsum = lt2;
        G->SoZ = (float)(G->S / Z);
        G->ticket = 0;
    }
}

// Kernel spectrum records of grid.cu (for (kx, ky) in [0, H)^2: K2, Ke, K1,
// Kln and D2x, Dex, D2y, Dey, 1/L^2 applied) repacked for the S2 epilogue:
// times the fold weights w_ky w_kx, with D = -Im of the odd kernels' spectra.
__global__ void k_dft_kpack(const GridDev* __restrict__ G, const float4* __restrict__ kc, float4* __restrict__ kp)
{
    const DftDims d = dft_dims(G);
    const int H = d.H;
    const int64_t tot = (int64_t)H * H;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < tot; u += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(u / H), ky = (int)(u - (int64_t)kx * H);
        const float w = ((ky == 0 || ky == H - 1) ? 1.0f : 2.0f) * ((kx == 0 || kx == H - 1) ? 1.0f : 2.0f);
        const float4 a = kc[2 * u], b = kc[2 * u + 1];
        kp[2 * u] = make_float4(a.x * w, a.y * w, a.z * w, a.w * w);
        kp[2 * u + 1] = make_float4(-b.x * w, -b.y * w, -b.z * w, -b.w * w);
    }
}

}  // namespace
}  // namespace lt

// ---- host side ----
namespace lt {
namespace {

struct DftSizes {
    int64_t F, G, W, X, Q, R;  // elements per split term
    int64_t K;                 // floats of the packed kernel table
    int64_t T;                 // floats of the S2 spectra
};

DftSizes dft_sizes(const IterShape& sh)
{
    const int64_t Mp = rup(sh.Mmax, 64), Kf = rup(2 * (sh.Lmax / 2 + 1), 64);
    DftSizes z;
    z.F = rup(Kf, 256) * Mp;
    z.G = rup(Mp, 256) * Kf;
    z.W = 4 * Mp * Mp;
    z.X = 4 * Kf * Mp;
    z.Q = 8 * Kf * Kf;
    z.R = 8 * Mp * Kf;
    z.K = 8 * (sh.Lmax / 2 + 1) * (int64_t)(sh.Lmax / 2 + 1);
    z.T = 4 * Kf * Kf;
    return z;
}

template <int ST, int BN>
cudaError_t set_gemm_attr()
{
    return cudaFuncSetAttribute(k_dft_gemm<ST, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gemm_smem_bytes<BN>());
}

// Tile widths of the four products (columns per tile).
constexpr int kBN1 = 128, kBN2 = 128, kBN4 = 128, kBN5 = 128;

}  // namespace

void dft_carve(Carve& c, const IterShape& sh, DftWs& w)
{
    const DftSizes z = dft_sizes(sh);
    w.pF = z.F; w.F = c.take<uint16_t>(kTerms * z.F);
    w.pG = z.G; w.G = c.take<uint16_t>(kTerms * z.G);
    w.pW = z.W; w.W = c.take<uint16_t>(kTerms * z.W);
    w.pX = z.X; w.X = c.take<uint16_t>(kTerms * z.X);
    w.pQ = z.Q; w.Q = c.take<uint16_t>(kTerms * z.Q);
    w.pR = z.R; w.R = c.take<uint16_t>(kTerms * z.R);
    w.kpack = c.take<float>(z.K);
    w.T = c.take<float>(z.T);
    w.tabM = c.take<int32_t>(1);
}

// No table is built yet; every other operand is rewritten, padding included,
// before it is read.
cudaError_t dft_reset(const DftWs& w, cudaStream_t s) { return cudaMemsetAsync(w.tabM, 0xFF, sizeof(int32_t), s); }

cudaError_t dft_set_attrs()
{
    cudaError_t e;
    if ((e = set_gemm_attr<1, kBN1>()) != cudaSuccess) return e;
    if ((e = set_gemm_attr<2, kBN2>()) != cudaSuccess) return e;
    if ((e = set_gemm_attr<3, kBN4>()) != cudaSuccess) return e;
    return set_gemm_attr<4, kBN5>();
}

cudaError_t launch_dft_prep(const IterWs& w, cudaStream_t s)
{
    const unsigned blocks = (unsigned)num_sms() * 4;
    k_dft_tables<<<blocks, 256, 0, s>>>(w.g, w.tw, w.dft);
    k_dft_charges<<<blocks, 256, 0, s>>>(w.g, w.wflt, w.dft, w.bcnt);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_dft_products(const IterWs& w, int32_t n, cudaStream_t s)
{
    k_dft_kpack<<<(unsigned)num_sms() * 4, 256, 0, s>>>(w.g, w.kc, (float4*)w.dft.kpack);
    GemmArgs a;
    a.G = w.g;
    a.st = w.st;
    a.w = w.dft;
    a.fields = w.fields;
    a.zblk = w.zblk;
    a.n = n;
    const unsigned grid = (unsigned)std::min(num_sms(), 512);  // persistent; S2's partial sums hold 512 blocks
    k_dft_gemm<1, kBN1><<<grid, kGemmThreads, gemm_smem_bytes<kBN1>(), s>>>(a);
    k_dft_gemm<2, kBN2><<<grid, kGemmThreads, gemm_smem_bytes<kBN2>(), s>>>(a);
    k_dft_products<<<(unsigned)std::min(num_sms() * 2, 512), kProdThreads, 0, s>>>(w.g, w.dft, (const float4*)w.dft.kpack,
                                                                                 w.st, w.zblk, n);
    k_dft_gemm<3, kBN4><<<grid, kGemmThreads, gemm_smem_bytes<kBN4>(), s>>>(a);
    k_dft_gemm<4, kBN5><<<grid, kGemmThreads, gemm_smem_bytes<kBN5>(), s>>>(a);
    count_launches(6);
    return cudaGetLastError();
}

}  // namespace lt
