// Internal: per-iteration device state of the interpolation grid and the
// launch helpers shared by grid.cu (spread, FFT convolution, Z) and
// iterate.cu (fused gather + attraction + compression + update).
#pragma once
#include "common.cuh"

namespace lt {

constexpr int kLMax = 4096;     // longest FFT line (L = 2 * P * I)
constexpr int kMaxRadix = 16;   // FFT stages
constexpr int kFieldStride = 8; // floats per grid node in the field array


// Written by k_setup every iteration from the layout bounds.  All integer
// decisions (I, box) are FP32 and match the oracle's grid rule bit for bit.
struct GridDev {
    float lo, hi, ext, h, s, c;  // domain [lo, lo+ext], box width h, node spacing s, centre c
    float rh, rs;                // 1/h and 1/s, correctly rounded
    int32_t I, M, L;             // boxes per dim, nodes per dim (I*P), FFT length (2M)
    int32_t P;                   // nodes per box
    int32_t nst;                 // FFT stages
    int32_t radix[kMaxRadix];
    float fx[4], ifx[4];         // 64-bit fixed-point scale per charge and its inverse (powers of 2)
    float hf[4], ihf[4];         // 32-bit per-point quantisation of warp-summed boxes
    double Z;                    // sum_{i != j} 1/(1+d^2), from the grid
    double S;                    // sum of P values
    double Lsum;                 // sum_{i,j} ln(eps + d^2) from the grid (self terms included)
    float SoZ;                   // S / Z rounded to FP32 (the repulsion scale)
    int32_t ticket;              // last-block counter for the Z reduction
    int32_t scan_ticket;         // last-block counter of the box scan
    int32_t nheavy;              // boxes summed by warps
    int32_t nitems;              // their segments
    int32_t imax;                // largest I of the run so far (cleared by iter_reset)
};

// Per-iteration scalars of the gradient, precomputed on the host in FP64:
// g = a_att A - a_rep (S/Z) R + a_cmp X - a_ent E.
struct Stage {
    float a_att;  // 4 lambda_KL alpha
    float a_rep;  // 4 lambda_KL
    float a_cmp;  // lambda_c / n
    float a_ent;  // lambda_r / n^2
    float momentum, lr;
};

// Split-BF16 operand matrices of the DFT-as-GEMM convolution (dftgemm.cu):
// the DFT tables F and G, the charges W, the x-transforms X, the kernel
// products Q and the inverse y-transforms R; each holds its BF16 split terms
// as consecutive planes of the stated number of elements.
struct DftWs {
    uint16_t *F, *G, *W, *X, *Q, *R;
    int64_t pF, pG, pW, pX, pQ, pR;  // elements per plane
    float* kpack;                    // kernel spectra packed for k_dft_products
    float* T;                        // FP32 spectra of the charges (S2 output)
    int32_t* tabM;                   // grid size the tables hold (-1: none)
};

// Device buffers of one gradient/optimize call, carved from the workspace.
struct IterWs {
    StatusBlock* st;
    GridDev* g;
    int32_t* bounds;     // [2 parities][2] ordered ints (min, max)
    float2* tw;          // twiddles e^{-2 pi i t/L}, kLMax
    int32_t* bcnt;       // max_boxes^2 points per box
    int32_t* bcur;       // max_boxes^2 block-local box offsets / scatter cursors
    int32_t* heavy;      // boxes summed by warps (G->nheavy of them)
    int32_t* hticket;    // per heavy box: segments finished
    long long* hacc;     // per heavy box: P^2 x 4 fixed-point sums
    int2* items;         // heavy-box segments (heavy index, segment)
    int32_t* btot;       // totals of the box-scan blocks
    int32_t* bpre;       // their exclusive scan
    float2* su;          // n local coordinates, box-sorted
    float4* wflt;        // M_max^2 float charges (plain form)
    float2* krow;        // 3 * H * H kernel row transforms [q][kx][a] (H = L_max/2 + 1)
    float4* kc;          // H * H records of 8 floats: kernel spectra (K2, Ke, K1, ln; D2x, Dex, D2y, Dey)
    float2* srow;        // 4 * M_max * H row half spectra of S0, S1x, S1y, S2
    float2* ucol;        // 6 * M_max * H column results
    float* fields;       // M_max^2 * 8
    double* zblk;        // per-block Z partials (DFT-GEMM products)
    double* zcol;        // per-column Z and entropy-sum terms of the FFT column pass
    double* sblk;        // per-block sum(P) partials
    float2* yalt;        // n, ping-pong layout
    float* phi;          // n * 8 (plain form gather output)
    float2* attr;        // n (plain form attraction output)
    DftWs dft;           // conv_mode 1 only (null pointers otherwise)
};

struct IterShape {
    int32_t n;
    int32_t P;
    int32_t max_boxes;
    int32_t Mmax, Lmax;
    int64_t hcap;  // capacity of the heavy-box lists
    int conv_mode;
};

// One graph of a batched run: its P, layouts, optimiser state, stage
// coefficients and iteration workspace.  The batched kernels serve every
// graph of a batch in one launch, graph = blockIdx.y, each graph's work
// split over gridDim.x blocks exactly as in a single-graph launch.
struct BatchGraph {
    IterWs w;
    const int64_t* P_row;
    const int32_t* P_col;
    const int16_t* P_d16;
    const float* P_val;
    float2* Y;  // the layout of parity 0 (w.yalt holds parity 1)
    float2* upd;
    float2* gains;
    Stage st;
    int32_t n;
    int32_t max_boxes;  // this graph's grid cap
    // rows of P summed in chunks before the fused kernel (nchunks = 0: none)
    const int32_t* hbase;
    const int32_t* crow;
    const int64_t* cstart;
    float2* hpartial;
    int32_t nchunks;
};

// Launch shape of the batched kernels (blocks per graph), chosen by the
// caller's tuning.
struct BatchShape {
    int32_t fft_blocks;     // FFT passes and kernel spectra
    int32_t spread_blocks;  // box spread
    int32_t max_n;          // largest graph (sizes the point-indexed grids)
};

IterShape iter_shape(int32_t n, const ltsnet_params* p);
IterWs iter_carve(Carve& c, const IterShape& sh);
cudaError_t iter_reset(const IterWs& w, const IterShape& sh, cudaStream_t s);

// Box of coordinate x: floor(RN(RN(x - lo) / h)) clamped to [0, I), the FP32
// operations of the oracle's grid rule.  d * rh (rh = RN(1/h)) is within a
// few units in the last place of RN(d / h), so its floor is the same unless it
// lies within 8 units of an integer, where the correctly rounded quotient
// decides.
__device__ __forceinline__ int box_of_r(float x, float lo, float h, float rh, int I)
{
    const float d = __fsub_rn(x, lo);
    float q = __fmul_rn(d, rh);
    float f = floorf(q);
    const float margin = fabsf(q) * 9.5367431640625e-7f;  // 2^-20: 8 units of q
    if (__fsub_rn(q, f) <= margin || __fsub_rn(__fadd_rn(f, 1.0f), q) <= margin) {
        q = __fdiv_rn(d, h);
        f = floorf(q);
    }
    const int b = (int)f;
    return b < 0 ? 0 : (b > I - 1 ? I - 1 : b);
}

// Lagrange weights at local coordinate u (in node spacings from the box's
// lower edge) for the P nodes of a box at u_a = a + 1/2.
template <int P>
__device__ __forceinline__ void lagrange(float u, float* w)
{
#pragma unroll
    for (int a = 0; a < P; ++a) {
        float num = 1.0f, den = 1.0f;
#pragma unroll
        for (int b = 0; b < P; ++b) {
            if (b == a) continue;
            num *= u - ((float)b + 0.5f);
            den *= (float)(a - b);
        }
        w[a] = num / den;
    }
}

// Round a float to the nearest 64-bit integer (ties to even) with integer
// operations only, from its sign, exponent and 24-bit significand.  Same
// result as a hardware float-to-int64 conversion for |x| < 2^62, which on
// this GPU would go through the narrow FP64 pipe.
__device__ __forceinline__ long long f2ll_rn(float x)
{
    const unsigned bits = __float_as_uint(x);
    const int e = (int)((bits >> 23) & 0xffu) - 127;  // unbiased exponent
    if (e < -1) return 0;                              // |x| < 0.5 (and zeros, denormals)
    const unsigned m = (bits & 0x7fffffu) | 0x800000u;  // significand, value = m * 2^(e - 23)
    long long r;
    if (e >= 23) {
        r = (long long)m << (e - 23);
    } else {
        const int sh = 23 - e;  // 1 .. 24
        const unsigned q = m >> sh, rem = m & ((1u << sh) - 1u), half = 1u << (sh - 1);
        r = (long long)(q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u));
    }
    return (bits >> 31) ? -r : r;
}

// Lagrange basis function a alone at local coordinate u.
template <int P>
__device__ __forceinline__ float lagrange_one(float u, int a)
{
    float num = 1.0f, den = 1.0f;
#pragma unroll
    for (int b = 0; b < P; ++b) {
        if (b == a) continue;
        num *= u - ((float)b + 0.5f);
        den *= (float)(a - b);
    }
    return num / den;
}

// (x - lo) / s - base to FP32 accuracy of the result itself, although
// (x - lo) / s can be in the thousands: x - lo is split exactly into
// d_hi + d_lo (TwoSum), q = d_hi / s is taken from the reciprocal rs = 1/s,
// its remainder d_hi - q s is formed with one rounding (FMA) and divided by
// s again, and q - base is exact (Sterbenz: base <= q <= 2 base, or base = 0),
// so the error of q does not reach the result beyond a unit or two of it.
__device__ __forceinline__ float local_u(float x, float lo, float s, float rs, int base)
{
    const float d_hi = __fsub_rn(x, lo);
    const float bb = __fsub_rn(d_hi, x);
    const float d_lo = __fadd_rn(__fsub_rn(x, __fsub_rn(d_hi, bb)), __fsub_rn(-lo, bb));
    const float q = __fmul_rn(d_hi, rs);
    const float r = __fmaf_rn(-q, s, d_hi);
    const float t_lo = __fmul_rn(__fadd_rn(r, d_lo), rs);
    return __fadd_rn(__fsub_rn(q, (float)base), t_lo);
}

// Box of a point and its local coordinates inside the box, in node spacings
// (u in [0, P]; the box's nodes sit at u = a + 1/2).
__device__ __forceinline__ void local_coords(float2 p, const GridDev* G, int& bx, int& by, float& ux, float& uy)
{
    const float lo = G->lo, h = G->h, s = G->s, rh = G->rh, rs = G->rs;
    const int I = G->I, P = G->P;
    bx = box_of_r(p.x, lo, h, rh, I);
    by = box_of_r(p.y, lo, h, rh, I);
    ux = local_u(p.x, lo, s, rs, P * bx);
    uy = local_u(p.y, lo, s, rs, P * by);
}

// order.cu
size_t order_ws_bytes(int32_t n);
cudaError_t bfs_order(const int64_t* row_ptr, const int32_t* col, int32_t n, int32_t* order, int32_t* inv, void* ws,
                      cudaStream_t s, bool* reordered);
cudaError_t permute_conditional_rows(const int32_t* order, const int32_t* inv, const int32_t* nbr,
                                     const double* pcond, const int32_t* cnt, int32_t n, int32_t k, int32_t* nbr2,
                                     double* pcond2, int32_t* cnt2, cudaStream_t s);
cudaError_t gather_rows2(const float2* src, const int32_t* idx, int32_t n, float2* dst, cudaStream_t s);

// grid.cu
cudaError_t launch_bounds_init(const IterWs& w, const float2* Y, int32_t n, int parity, cudaStream_t s);
cudaError_t launch_psum(const IterWs& w, const int64_t* P_row, int32_t n, const float* P_val, cudaStream_t s);
cudaError_t grid_set_smem_attrs();
// dftgemm.cu
void dft_carve(Carve& c, const IterShape& sh, DftWs& w);
cudaError_t dft_reset(const DftWs& w, cudaStream_t s);
cudaError_t dft_set_attrs();
cudaError_t launch_dft_prep(const IterWs& w, cudaStream_t s);
cudaError_t launch_dft_products(const IterWs& w, int32_t n, cudaStream_t s);
cudaError_t launch_grid_phase(const IterWs& w, const IterShape& sh, const ltsnet_params* p, const float2* Y,
                              int parity, bool plain, cudaStream_t s);
cudaError_t launch_grid_phase_batched(const BatchGraph* bg, int32_t ng, const BatchShape& bs, const IterShape& sh,
                                      const ltsnet_params* p, int parity, cudaStream_t s);

}  // namespace lt
