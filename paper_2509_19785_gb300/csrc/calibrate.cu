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
// This group-per-row form serves k > kTileK; k_calibrate_rows below the rest.
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

// Thread-per-row form for k <= kTileK (the common case).  GB300's FP64 rate is
// a small fraction of its FP32 rate, so each search step first evaluates H in
// FP32; only when that value lies within tol + kH32Margin of ln u (where the
// FP32 error could change the decision) is H evaluated in FP64.  Outside that
// band the FP64 value is on the same side of ln u and farther than tol from
// it, so the sequence of beta values, the stopping step and the result are
// those of the all-FP64 search.  A warp's 32 hop rows are staged in shared
// memory with coalesced loads, and its 32 output rows written coalesced; the
// output values come from one exp per shell.
constexpr int kCalThreads = 128;
constexpr int kShells = 16;
constexpr int kTileK = 512;
constexpr float kH32Margin = 1e-4f;

__device__ __forceinline__ double shell_entropy64(const uint16_t* hv, const uint16_t* nv, int R, double dmin,
                                                  double beta, double& S)
{
    double D = 0.0;
    S = 0.0;
    for (int r = 0; r < R; ++r) {
        const double dd = (double)hv[r] * (double)hv[r] - dmin;
        const double cw = (double)nv[r] * exp(-beta * dd);
        S += cw;
        D += cw * dd;
    }
    return log(S) + beta * D / S;
}

__global__ void __launch_bounds__(kCalThreads)
    k_calibrate_rows(const uint16_t* __restrict__ hop, const int32_t* __restrict__ cnt, int32_t n, int32_t k,
                     double target, double tol, int32_t max_steps, double* __restrict__ beta_out,
                     double* __restrict__ pcond, uint8_t* __restrict__ conv)
{
    extern __shared__ __align__(16) unsigned char cal_smem[];
    uint16_t* tile = (uint16_t*)cal_smem;  // [kCalThreads][k]
    __shared__ uint16_t sh_h[kCalThreads][kShells];
    __shared__ uint16_t sh_n[kCalThreads][kShells];
    __shared__ double sh_e[kCalThreads][kShells];
    __shared__ int sh_R[kCalThreads];
    __shared__ int sh_c[kCalThreads];
    const int t = threadIdx.x, lane = t & 31, wb = t & ~31;
    const float tgt32 = (float)target;
    for (int64_t base = (int64_t)blockIdx.x * kCalThreads; base < n; base += (int64_t)gridDim.x * kCalThreads) {
        // stage the warp's 32 hop rows (contiguous in memory)
        const int64_t wrow0 = base + wb;
        const int wrows = (int)min((int64_t)32, max((int64_t)0, (int64_t)n - wrow0));
        {
            const uint16_t* src = hop + wrow0 * (int64_t)k;
            uint16_t* dst = tile + (int64_t)wb * k;
            for (int i = lane; i < wrows * k; i += 32) dst[i] = src[i];
        }
        __syncwarp();
        const int64_t row = base + t;
        const uint16_t* h = tile + (int64_t)t * k;
        int c = 0, R = 0;
        double beta = 1.0, S = 1.0;
        bool ok = false;
        if (row < n) {
            c = min(cnt[row], k);
            int prev = -1;
            for (int j = 0; j < c; ++j) {
                const int hv = h[j];
                if (hv != prev) {
                    if (R < kShells) {
                        sh_h[t][R] = (uint16_t)hv;
                        sh_n[t][R] = 0;
                    }
                    ++R;
                    prev = hv;
                }
                if (R <= kShells) sh_n[t][R - 1] += 1;
            }
        }
        const bool shells = R <= kShells;
        if (row < n && c > 0) {
            int hmin = 0x7fffffff;
            if (shells)
                for (int r = 0; r < R; ++r) hmin = min(hmin, (int)sh_h[t][r]);
            else
                for (int j = 0; j < c; ++j) hmin = min(hmin, (int)h[j]);
            const double dmin = (double)hmin * (double)hmin;
            double lo = -INFINITY, hi = INFINITY;
            for (int step = 0; step < max_steps; ++step) {
                double diff;
                bool exact = !shells || !(beta > 1e-20 && beta < 1e20);
                if (!exact) {
                    const float bf = (float)beta;
                    float Sf = 0.f, Df = 0.f;
                    for (int r = 0; r < R; ++r) {
                        const float dd = (float)((int)sh_h[t][r] * (int)sh_h[t][r] - hmin * hmin);
                        const float cw = (float)sh_n[t][r] * expf(-bf * dd);
                        Sf += cw;
                        Df += cw * dd;
                    }
                    const float d32 = logf(Sf) + bf * Df / Sf - tgt32;
                    if (fabsf(d32) > (float)tol + kH32Margin && isfinite(d32)) diff = (double)d32;
                    else exact = true;
                }
                if (exact) {
                    double H;
                    if (shells) {
                        H = shell_entropy64(sh_h[t], sh_n[t], R, dmin, beta, S);
                    } else {
                        double Sx = 0.0, D = 0.0;
                        for (int j = 0; j < c; ++j) {
                            const double dd = (double)h[j] * (double)h[j] - dmin;
                            const double w = exp(-beta * dd);
                            Sx += w;
                            D += w * dd;
                        }
                        H = log(Sx) + beta * D / Sx;
                    }
                    diff = H - target;
                    if (fabs(diff) < tol) {
                        ok = true;
                        break;
                    }
                }
                if (diff > 0.0) {
                    lo = beta;
                    beta = (hi == INFINITY) ? beta * 2.0 : (beta + hi) / 2.0;
                } else {
                    hi = beta;
                    beta = (lo == -INFINITY) ? beta / 2.0 : (beta + lo) / 2.0;
                }
            }
            // normaliser and per-shell probabilities at the final beta
            if (shells) {
                S = 0.0;
                for (int r = 0; r < R; ++r)
                    S += (double)sh_n[t][r] * exp(-beta * ((double)sh_h[t][r] * (double)sh_h[t][r] - dmin));
                for (int r = 0; r < R; ++r)
                    sh_e[t][r] = exp(-beta * ((double)sh_h[t][r] * (double)sh_h[t][r] - dmin)) / S;
            } else {
                S = 0.0;
                for (int j = 0; j < c; ++j) S += exp(-beta * ((double)h[j] * (double)h[j] - dmin));
            }
            sh_R[t] = shells ? R : -1;
            sh_c[t] = c;
            beta_out[row] = beta;
            conv[row] = ok ? 1 : 0;
            sh_e[t][0] = shells ? sh_e[t][0] : S;  // the normaliser, for the per-neighbour output
            if (!shells) sh_h[t][0] = (uint16_t)hmin;
        } else if (row < n) {
            sh_R[t] = 0;
            sh_c[t] = 0;
            beta_out[row] = 1.0;
            conv[row] = 0;
        }
        __syncwarp();
        // coalesced output of the warp's rows
        for (int r = 0; r < wrows; ++r) {
            const int tr = wb + r;
            const int Rr = sh_R[tr], cr = sh_c[tr];
            const uint16_t* hr = tile + (int64_t)tr * k;
            double* dst = pcond + (wrow0 + r) * (int64_t)k;
            for (int j = lane; j < k; j += 32) {
                double v = 0.0;
                if (j < cr) {
                    const int hv = hr[j];
                    if (Rr >= 0) {
                        for (int q = 0; q < Rr; ++q)
                            if ((int)sh_h[tr][q] == hv) {
                                v = sh_e[tr][q];
                                break;
                            }
                    } else {
                        const double dmin = (double)sh_h[tr][0] * (double)sh_h[tr][0];
                        v = exp(-beta_out[wrow0 + r] * ((double)hv * (double)hv - dmin)) / sh_e[tr][0];
                    }
                }
                dst[j] = v;
            }
        }
        __syncwarp();
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
    if (k <= kTileK) {
        const size_t smem = (size_t)kCalThreads * k * sizeof(uint16_t);
        LT_CUDA(once_per_device(kOnceCalib, [] {
            return cudaFuncSetAttribute(k_calibrate_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((size_t)kCalThreads * kTileK * sizeof(uint16_t)));
        }));
        int64_t blocks = ((int64_t)n + kCalThreads - 1) / kCalThreads;
        const int64_t cap = (int64_t)num_sms() * 16;
        if (blocks > cap) blocks = cap;
        k_calibrate_rows<<<(unsigned)blocks, kCalThreads, smem, (cudaStream_t)stream>>>(
            hop, cnt, n, k, log(perplexity), tol, max_steps, beta, pcond, converged);
    } else {
        int64_t blocks = ((int64_t)n + kRowsPerBlock - 1) / kRowsPerBlock;
        const int64_t cap = (int64_t)num_sms() * 16;
        if (blocks > cap) blocks = cap;
        k_calibrate<<<(unsigned)blocks, kGroup * kRowsPerBlock, 0, (cudaStream_t)stream>>>(
            hop, cnt, n, k, log(perplexity), tol, max_steps, beta, pcond, converged);
    }
    LT_CHECK_LAUNCH();
    count_launches(1);
    return LTSNET_OK;
}
