// K2 -- perplexity calibration in FP64 (Eq. 3 and the perplexity definition
// beneath it).
//
// The hop distances of a row are non-decreasing (BFS discovery order), so a
// row is a few "shells" of equal distance.  Each row is handled by a group of
// 8 lanes (4 rows per warp): the group compresses the row into (d^2, count)
// shells in shared memory, then runs the beta search evaluating
//   S(beta) = sum_r c_r exp(-beta (d_r^2 - d_min^2)),
//   H(beta) = ln S + beta * sum_r c_r (d_r^2 - d_min^2) exp(...) / S,
// which is -sum_j p_j ln p_j of Eq. 3 written per shell, with one exp per
// shell instead of one per neighbour.  The search steps are those of the
// method: start at beta = 1, double/halve until the target ln u is bracketed,
// then bisect, stop at |H - ln u| < tol or after max_steps evaluations.
// Rows with more than kMaxShells shells evaluate the sums per neighbour.
#include <math.h>

#include "common.cuh"

namespace lt {
namespace {

constexpr int kGroup = 8;          // lanes per row
constexpr int kRowsPerBlock = 16;  // 128 threads
constexpr int kMaxShells = 64;

__global__ void __launch_bounds__(kGroup* kRowsPerBlock)
    k_calibrate(const uint16_t* __restrict__ hop, const int32_t* __restrict__ cnt, int32_t n, int32_t k,
                double target, double tol, int32_t max_steps, double* __restrict__ beta_out,
                double* __restrict__ pcond, uint8_t* __restrict__ conv)
{
    __shared__ int32_t sh_d2[kRowsPerBlock][kMaxShells];
    __shared__ int32_t sh_start[kRowsPerBlock][kMaxShells + 1];
    const int g = threadIdx.x / kGroup;
    const int gl = threadIdx.x % kGroup;
    const int wl = threadIdx.x & 31;
    const int gbase = wl & ~(kGroup - 1);
    const unsigned gmask = 0xffu << gbase;

    for (int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + g; row < n;
         row += (int64_t)gridDim.x * kRowsPerBlock) {
        const int c = min(cnt[row], k);
        const uint16_t* h = hop + row * (int64_t)k;
        double* p = pcond + row * (int64_t)k;
        if (c <= 0) {
            for (int j = gl; j < k; j += kGroup) p[j] = 0.0;
            if (gl == 0) {
                beta_out[row] = 1.0;
                conv[row] = 0;
            }
            continue;
        }
        // Shell boundaries in order.
        int R = 0;
        for (int j0 = 0; j0 < c; j0 += kGroup) {
            const int j = j0 + gl;
            bool bnd = false;
            int hv = 0;
            if (j < c) {
                hv = h[j];
                bnd = (j == 0) || (h[j - 1] != hv);
            }
            const unsigned bal = (__ballot_sync(gmask, bnd) >> gbase) & 0xffu;
            const int idx = R + __popc(bal & ((1u << gl) - 1u));
            if (bnd && idx < kMaxShells) {
                sh_d2[g][idx] = hv * hv;
                sh_start[g][idx] = j;
            }
            R += __popc(bal);
        }
        const bool by_shell = R <= kMaxShells;
        if (by_shell && gl == 0) sh_start[g][R] = c;
        __syncwarp(gmask);
        int hmin = 0x7fffffff;
        for (int j = gl; j < c; j += kGroup) hmin = min(hmin, (int)h[j]);
#pragma unroll
        for (int o = kGroup / 2; o > 0; o >>= 1) hmin = min(hmin, __shfl_xor_sync(gmask, hmin, o));
        const double dmin = (double)hmin * (double)hmin;

        double beta = 1.0, lo = -INFINITY, hi = INFINITY;
        bool ok = false;
        for (int step = 0; step < max_steps; ++step) {
            double S = 0.0, D = 0.0;
            if (by_shell) {
                for (int r = gl; r < R; r += kGroup) {
                    const double dd = (double)sh_d2[g][r] - dmin;
                    const double cw = (double)(sh_start[g][r + 1] - sh_start[g][r]) * exp(-beta * dd);
                    S += cw;
                    D += cw * dd;
                }
            } else {
                for (int j = gl; j < c; j += kGroup) {
                    const double dd = (double)h[j] * (double)h[j] - dmin;
                    const double w = exp(-beta * dd);
                    S += w;
                    D += w * dd;
                }
            }
#pragma unroll
            for (int o = kGroup / 2; o > 0; o >>= 1) {
                S += __shfl_xor_sync(gmask, S, o);
                D += __shfl_xor_sync(gmask, D, o);
            }
            const double H = log(S) + beta * D / S;
            const double diff = H - target;
            if (fabs(diff) < tol) {
                ok = true;
                break;
            }
            if (diff > 0.0) {
                lo = beta;
                beta = (hi == INFINITY) ? beta * 2.0 : (beta + hi) / 2.0;
            } else {
                hi = beta;
                beta = (lo == -INFINITY) ? beta / 2.0 : (beta + lo) / 2.0;
            }
        }
        // p_{j|i} at the final beta.
        double S = 0.0;
        if (by_shell) {
            for (int r = gl; r < R; r += kGroup)
                S += (double)(sh_start[g][r + 1] - sh_start[g][r]) * exp(-beta * ((double)sh_d2[g][r] - dmin));
        } else {
            for (int j = gl; j < c; j += kGroup) S += exp(-beta * ((double)h[j] * (double)h[j] - dmin));
        }
#pragma unroll
        for (int o = kGroup / 2; o > 0; o >>= 1) S += __shfl_xor_sync(gmask, S, o);
        for (int j = gl; j < k; j += kGroup)
            p[j] = (j < c) ? exp(-beta * ((double)h[j] * (double)h[j] - dmin)) / S : 0.0;
        if (gl == 0) {
            beta_out[row] = beta;
            conv[row] = ok ? 1 : 0;
        }
        __syncwarp(gmask);
    }
}

}  // namespace
}  // namespace lt

extern "C" ltsnet_status ltsnet_calibrate(const uint16_t* hop, const int32_t* cnt, int32_t n, int32_t k,
                                          double perplexity, double tol, int32_t max_steps, double* beta,
                                          double* pcond, uint8_t* converged, ltsnet_stream stream)
{
    using namespace lt;
    if (n < 0 || k < 1 || k > LTSNET_MAX_K || !(perplexity > 0.0) || !(tol > 0.0) || max_steps < 1)
        return LTSNET_ERR_INVALID_ARG;
    if (n == 0) return LTSNET_OK;
    if (!hop || !cnt || !beta || !pcond || !converged) return LTSNET_ERR_INVALID_ARG;
    int64_t blocks = ((int64_t)n + kRowsPerBlock - 1) / kRowsPerBlock;
    const int64_t cap = (int64_t)kSMs * 16;
    if (blocks > cap) blocks = cap;
    k_calibrate<<<(unsigned)blocks, kGroup * kRowsPerBlock, 0, (cudaStream_t)stream>>>(
        hop, cnt, n, k, log(perplexity), tol, max_steps, beta, pcond, converged);
    LT_CHECK_LAUNCH();
    count_launches(1);
    return LTSNET_OK;
}
