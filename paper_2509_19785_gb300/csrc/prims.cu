// Device-wide exclusive scan and stable LSD radix sort (used by the
// symmetrisation step).  Reduce-then-scan: per-tile sums, a single-block scan
// of the tile sums, then per-tile scans with the tile's offset.  The radix
// sort keeps stability by giving each warp a contiguous sub-tile and ranking
// keys inside a warp with __match_any_sync in input order.
#include "prims.cuh"

namespace lt {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot, uint32_t& excl)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? warp_tot[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(FULL, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < nw) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == 31) warp_tot[32] = ti;       // block total
    }
    __syncthreads();
    excl = warp_tot[w] + inc - v;
    uint32_t total = warp_tot[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, int64_t count,
                                                              uint32_t* __restrict__ bsum)
{
    __shared__ uint32_t wt[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < count) s += in[base + i];
    uint32_t ex;
    uint32_t tot = block_exclusive_scan(s, wt, ex);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t* __restrict__ bsum, int64_t nb)
{
    __shared__ uint32_t wt[33];
    uint32_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += kScanTile) {
        const int64_t base = c0 + (int64_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = (base + i < nb) ? bsum[base + i] : 0u;
            s += v[i];
        }
        uint32_t ex;
        uint32_t tot = block_exclusive_scan(s, wt, ex);
        uint32_t run = carry + ex;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (base + i < nb) bsum[base + i] = run;
            run += v[i];
        }
        carry += tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, uint32_t* out, int64_t count,
                                                            const uint32_t* __restrict__ bsum)
{
    __shared__ uint32_t wt[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < count) ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t ex;
    block_exclusive_scan(s, wt, ex);
    uint32_t run = bsum[blockIdx.x] + ex;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < count) out[base + i] = run;
        run += v[i];
    }
}

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixItems = 16;  // per lane
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kDigits = 256;

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint64_t* __restrict__ keys, int64_t count,
                                                              int shift, uint32_t* __restrict__ hist, int64_t nblocks)
{
    __shared__ uint32_t c[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kRadixThreads) c[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll 4
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t e = base + (int64_t)i * kRadixThreads + threadIdx.x;
        if (e < count) atomicAdd(&c[(unsigned)(keys[e] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += kRadixThreads) hist[(int64_t)d * nblocks + blockIdx.x] = c[d];
}

// Stable scatter of one tile: per-warp digit counts, then every key's place
// inside the tile (digit-major, input order within a digit) in shared
// memory, then the tile is written out in that order, so each digit's run
// goes to global memory as consecutive addresses.
constexpr size_t kScatterSmem = (size_t)kRadixTile * (sizeof(uint64_t) + sizeof(double));
constexpr size_t kScatterSmemKeys = (size_t)kRadixTile * sizeof(uint64_t);  // keys alone

// VALS: (key, value) pairs, else keys alone (vin, vout unused).
template <bool VALS>
__global__ void __launch_bounds__(kRadixThreads, 2)
    k_radix_scatter(const uint64_t* __restrict__ kin, const double* __restrict__ vin, uint64_t* __restrict__ kout,
                    double* __restrict__ vout, int64_t count, int shift, const uint32_t* __restrict__ offs,
                    int64_t nblocks)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t* sk = (uint64_t*)rs_smem;
    double* sv = (double*)(sk + kRadixTile);
    __shared__ uint32_t wh[kRadixWarps][kDigits];
    __shared__ uint32_t dstart[kDigits];  // first tile-local place of each digit
    __shared__ uint32_t gbase[kDigits];   // global place of each digit's first key of this tile
    __shared__ uint32_t wt[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned ltm = lanemask_lt();
    for (int d = lane; d < kDigits; d += 32) wh[w][d] = 0;
    __syncwarp();
    const int64_t tile0 = (int64_t)blockIdx.x * kRadixTile;
    const int64_t base = tile0 + (int64_t)w * (32 * kRadixItems);
    uint64_t kk[kRadixItems];
    double vv[kRadixItems];
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t e = base + i * 32 + lane;
        if (e < count) {
            kk[i] = kin[e];
            if (VALS) vv[i] = vin[e];
        }
    }
    // per-warp digit counts over the warp's sub-tile
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t e = base + i * 32 + lane;
        const bool valid = e < count;
        const int d = valid ? (int)((kk[i] >> shift) & 0xffu) : -1;
        const unsigned peers = __match_any_sync(FULL, d);
        if (valid && (peers & ltm) == 0) wh[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // tile totals per digit, their exclusive scan, and the warps' offsets
    uint32_t tot = 0;
    if (threadIdx.x < kDigits)
        for (int ww = 0; ww < kRadixWarps; ++ww) tot += wh[ww][threadIdx.x];
    uint32_t start = 0;
    block_exclusive_scan(threadIdx.x < kDigits ? tot : 0u, wt, start);
    if (threadIdx.x < kDigits) {
        const int d = threadIdx.x;
        dstart[d] = start;
        gbase[d] = offs[(int64_t)d * nblocks + blockIdx.x];
        uint32_t run = start;
        for (int ww = 0; ww < kRadixWarps; ++ww) {
            const uint32_t c = wh[ww][d];
            wh[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    // tile-local places, input order within a digit
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t e = base + i * 32 + lane;
        const bool valid = e < count;
        const int d = valid ? (int)((kk[i] >> shift) & 0xffu) : -1;
        const unsigned peers = __match_any_sync(FULL, d);
        if (valid) {
            const uint32_t lp = wh[w][d] + __popc(peers & ltm);
            sk[lp] = kk[i];
            if (VALS) sv[lp] = vv[i];
        }
        __syncwarp();
        if (valid && (peers & ltm) == 0) wh[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    const int nt = (int)min((int64_t)kRadixTile, count - tile0);
    for (int j = threadIdx.x; j < nt; j += kRadixThreads) {
        const uint64_t key = sk[j];
        const int d = (int)((key >> shift) & 0xffu);
        const uint32_t gp = gbase[d] + ((uint32_t)j - dstart[d]);
        kout[gp] = key;
        if (VALS) vout[gp] = sv[j];
    }
}

}  // namespace

size_t scan_tmp_words(int64_t count)
{
    int64_t nb = (count + kScanTile - 1) / kScanTile;
    return (size_t)(nb > 0 ? nb : 1);
}

cudaError_t scan_u32_exclusive(const uint32_t* in, uint32_t* out, int64_t count, uint32_t* tmp, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int64_t nb = (count + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, count, tmp);
    k_scan_top<<<1, kScanThreads, 0, s>>>(tmp, nb);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, count, tmp);
    count_launches(3);
    return cudaGetLastError();
}

size_t radix_hist_words(int64_t count)
{
    int64_t nb = (count + kRadixTile - 1) / kRadixTile;
    return (size_t)(nb > 0 ? nb : 1) * kDigits;
}

cudaError_t radix_sort_u64_f64(uint64_t* k0, double* v0, uint64_t* k1, double* v1, int64_t count, int bits,
                               uint32_t* hist, uint32_t* tmp, cudaStream_t s, bool* in_alt)
{
    *in_alt = false;
    if (count <= 1) return cudaSuccess;
    const int64_t nb = (count + kRadixTile - 1) / kRadixTile;
    {
        cudaError_t e = once_per_device(kOnceRadix, [] {
            return cudaFuncSetAttribute(k_radix_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kScatterSmem);
        });
        if (e != cudaSuccess) return e;
    }
    uint64_t *ka = k0, *kb = k1;
    double *va = v0, *vb = v1;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nb, kRadixThreads, 0, s>>>(ka, count, shift, hist, nb);
        count_launches(1);
        cudaError_t e = scan_u32_exclusive(hist, hist, nb * kDigits, tmp, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<true><<<(unsigned)nb, kRadixThreads, kScatterSmem, s>>>(ka, va, kb, vb, count, shift, hist,
                                                                                nb);
        count_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t* tk = ka; ka = kb; kb = tk;
        double* tv = va; va = vb; vb = tv;
        *in_alt = !*in_alt;
    }
    return cudaSuccess;
}

cudaError_t radix_sort_u64(uint64_t* k0, uint64_t* k1, int64_t count, int lo_bit, int bits, uint32_t* hist,
                           uint32_t* tmp, cudaStream_t s, bool* in_alt)
{
    *in_alt = false;
    if (count <= 1) return cudaSuccess;
    const int64_t nb = (count + kRadixTile - 1) / kRadixTile;
    uint64_t *ka = k0, *kb = k1;
    for (int shift = lo_bit; shift < lo_bit + bits; shift += 8) {
        k_radix_hist<<<(unsigned)nb, kRadixThreads, 0, s>>>(ka, count, shift, hist, nb);
        count_launches(1);
        cudaError_t e = scan_u32_exclusive(hist, hist, nb * kDigits, tmp, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<false><<<(unsigned)nb, kRadixThreads, kScatterSmemKeys, s>>>(ka, nullptr, kb, nullptr, count,
                                                                                    shift, hist, nb);
        count_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t* tk = ka; ka = kb; kb = tk;
        *in_alt = !*in_alt;
    }
    return cudaSuccess;
}

}  // namespace lt
