// K3 -- symmetrisation (Eq. 2): p_ij = (p_{j|i} + p_{i|j}) / (2n).
//
// Every conditional entry (i, j, p_{j|i}) at slot s of row i's list is
// emitted twice, as the 64-bit key (row i, col j, slot s, copy 0) and as
// (row j, col i, slot s, copy 1); padded slots get the key ~0, which sorts
// last.  A stable radix sort of the keys alone by their (row, col) bits
// brings the (at most two) copies of each pair together with rows and
// columns ascending; a head-flag scan numbers the distinct pairs; the write
// pass reads each copy's p_{j|i} back from its source's conditional row (row
// i for copy 0, column i for copy 1, slot s), adds the two in FP64, scales by
// 1/(2n), rounds once to FP32 and fills the CSR row offsets (including empty
// rows).  The key needs 2 ceil(log2(n + 1)) + ceil(log2 k) + 1 bits, which
// is at most 64 whenever the 2 n k emitted entries have 32-bit offsets.
// Scratch: two key buffers, 16 bytes per emitted entry; the head flags and
// pair numbers go into the key buffer the sort has left free.
#include "prims.cuh"

namespace lt {
namespace {

__global__ void k_sym_emit(const int32_t* __restrict__ nbr, const int32_t* __restrict__ cnt, int32_t n, int32_t k,
                             int nbits, int pb, uint64_t* __restrict__ keys, StatusBlock* st)
{
    const int64_t nk = (int64_t)n * k;
    const uint64_t tflag = 1ull << (pb - 1);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int s = (int)(e - i * k);
        uint64_t ko = ~0ull, kt = ~0ull;
        if (s < cnt[i]) {
            const int32_t v = nbr[e];
            if ((unsigned)v < (unsigned)n) {
                ko = ((((uint64_t)i << nbits) | (uint64_t)v) << pb) | (uint64_t)s;
                kt = ((((uint64_t)v << nbits) | (uint64_t)i) << pb) | tflag | (uint64_t)s;
            } else {
                record_error(st, LTSNET_ERR_BAD_GRAPH, v);
            }
        }
        keys[e] = ko;
        keys[nk + e] = kt;
    }
}

__global__ void k_sym_heads(const uint64_t* __restrict__ keys, int64_t E, int pb, uint32_t* __restrict__ flag)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = keys[e];
        flag[e] = (x != ~0ull && (e == 0 || (keys[e - 1] >> pb) != (x >> pb))) ? 1u : 0u;
    }
}

// p_{j|i} of a key: slot s of the source's conditional row, the
// source being the row, or the column for a transposed copy.
__device__ __forceinline__ double pair_p(uint64_t x, const double* __restrict__ pcond, int32_t k, int nbits,
                                            int pb)
{
    const uint64_t rc = x >> pb;
    const uint64_t cmask = (1ull << nbits) - 1ull;
    const bool tr = (x >> (pb - 1)) & 1ull;
    const int64_t src = tr ? (int64_t)(rc & cmask) : (int64_t)(rc >> nbits);
    const int64_t s = (int64_t)(x & ((1ull << (pb - 1)) - 1ull));
    return pcond[src * k + s];
}

__global__ void k_sym_write(const uint64_t* __restrict__ keys, const double* __restrict__ pcond,
                              const uint32_t* __restrict__ flag, const uint32_t* __restrict__ uidx, int64_t E,
                              int nbits, int pb, int32_t n, int32_t k, int64_t cap, double inv2n,
                              int64_t* __restrict__ P_row, int32_t* __restrict__ P_col, float* __restrict__ P_val,
                              int64_t* __restrict__ nnz_out)
{
    const uint64_t cmask = (1ull << nbits) - 1ull;
    const int rs = nbits + pb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[e]) continue;
        const uint64_t x = keys[e];
        const int64_t u = uidx[e];
        const int64_t row = (int64_t)(x >> rs);
        double v = pair_p(x, pcond, k, nbits, pb);
        const bool dup = (e + 1 < E) && (keys[e + 1] >> pb) == (x >> pb);
        if (dup) v = v + pair_p(keys[e + 1], pcond, k, nbits, pb);
        if (u < cap) {
            P_col[u] = (int32_t)((x >> pb) & cmask);
            P_val[u] = (float)(v * inv2n);
        }
        const int64_t prev_row = (e == 0) ? -1 : (int64_t)(keys[e - 1] >> rs);
        if (e == 0 || prev_row != row)
            for (int64_t r = prev_row + 1; r <= row; ++r) P_row[r] = u;
        const int64_t nxt = e + (dup ? 2 : 1);
        if (nxt >= E || keys[nxt] == ~0ull) {
            for (int64_t r = row + 1; r <= n; ++r) P_row[r] = u + 1;
            *nnz_out = u + 1;
        }
    }
}

__global__ void k_fill_i64(int64_t* p, int64_t count, int64_t v)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = v;
}

int sym_nbits(int32_t n)
{
    int b = 1;
    while (((int64_t)1 << b) < (int64_t)n + 1) ++b;
    return b;
}

// Bits of the key below (row, col): the slot in the source's list and the
// transposed-copy flag.
int sym_pbits(int32_t k)
{
    int b = 1;
    while (((int64_t)1 << b) < (int64_t)k) ++b;
    return b + 1;
}

bool sym_key_fits(int32_t n, int32_t k) { return 2 * sym_nbits(n) + sym_pbits(k) <= 64; }

struct SymWs {
    StatusBlock* st;
    uint64_t *k0, *k1;
    uint32_t *hist, *tmp;
    int64_t* nnz;
};

SymWs sym_carve(Carve& c, int32_t n, int32_t k)
{
    const int64_t E = 2 * (int64_t)n * k;
    SymWs w;
    w.st = c.take<StatusBlock>(1);
    w.nnz = c.take<int64_t>(1);
    w.k0 = c.take<uint64_t>(E);
    w.k1 = c.take<uint64_t>(E);
    const size_t hw = radix_hist_words(E);
    w.hist = c.take<uint32_t>(hw);
    size_t tw = scan_tmp_words(E);
    size_t tw2 = scan_tmp_words((int64_t)hw);
    w.tmp = c.take<uint32_t>(tw > tw2 ? tw : tw2);
    return w;
}

}  // namespace

int64_t symmetrize_max_nnz(int32_t n, int32_t k) { return 2 * (int64_t)n * k; }

}  // namespace lt

extern "C" int64_t ltsnet_symmetrize_max_nnz(int32_t n, int32_t k)
{
    if (n < 0 || k < 1) return 0;
    return lt::symmetrize_max_nnz(n, k);
}

extern "C" size_t ltsnet_symmetrize_workspace_size(int32_t n, int32_t k)
{
    if (n < 0 || k < 1) return 0;
    lt::Carve c(nullptr, 0);
    lt::sym_carve(c, n, k);
    return lt::align_up(c.off, 256);
}

extern "C" ltsnet_status ltsnet_symmetrize(const int32_t* nbr, const int32_t* cnt, const double* pcond, int32_t n,
                                           int32_t k, int64_t* P_row, int32_t* P_col, float* P_val, int64_t cap,
                                           int64_t* nnz_out, void* ws, size_t ws_bytes, ltsnet_stream stream)
{
    using namespace lt;
    if (n < 0 || k < 1 || k > LTSNET_MAX_K || cap < 0 || !nnz_out) return LTSNET_ERR_INVALID_ARG;
    *nnz_out = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        if (P_row) LT_CUDA(cudaMemsetAsync(P_row, 0, sizeof(int64_t), s));
        return LTSNET_OK;
    }
    if (!nbr || !cnt || !pcond || !P_row || (cap > 0 && (!P_col || !P_val)) || !ws) return LTSNET_ERR_INVALID_ARG;
    const int64_t E = 2 * (int64_t)n * k;
    if (E >= ((int64_t)1 << 32)) return LTSNET_ERR_INVALID_ARG;  // 32-bit scan offsets
    if ((uintptr_t)ws & 255) return LTSNET_ERR_WORKSPACE;
    Carve c(ws, ws_bytes);
    SymWs w = sym_carve(c, n, k);
    if (!c.ok()) return LTSNET_ERR_WORKSPACE;
    const int nbits = sym_nbits(n);
    if (!sym_key_fits(n, k)) return LTSNET_ERR_INVALID_ARG;  // not reached while E < 2^32
    const unsigned grid = num_sms() * 8, block = 256;
    LT_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StatusBlock), s));
    LT_CUDA(cudaMemsetAsync(w.nnz, 0, sizeof(int64_t), s));
    const int pb = sym_pbits(k);
    k_sym_emit<<<grid, block, 0, s>>>(nbr, cnt, n, k, nbits, pb, w.k0, w.st);
    LT_CHECK_LAUNCH();
    count_launches(1);
    bool alt = false;
    LT_CUDA(radix_sort_u64(w.k0, w.k1, E, pb, 2 * nbits, w.hist, w.tmp, s, &alt));
    const uint64_t* ks = alt ? w.k1 : w.k0;
    // head flags and pair numbers in the other key buffer, free after the sort
    uint32_t* flag = (uint32_t*)(alt ? w.k0 : w.k1);
    uint32_t* uidx = flag + E;
    k_sym_heads<<<grid, block, 0, s>>>(ks, E, pb, flag);
    LT_CHECK_LAUNCH();
    count_launches(1);
    LT_CUDA(scan_u32_exclusive(flag, uidx, E, w.tmp, s));
    k_fill_i64<<<64, 256, 0, s>>>(P_row, (int64_t)n + 1, 0);
    LT_CHECK_LAUNCH();
    count_launches(1);
    k_sym_write<<<grid, block, 0, s>>>(ks, pcond, flag, uidx, E, nbits, pb, n, k, cap, 1.0 / (2.0 * (double)n),
                                         P_row, P_col, P_val, w.nnz);
    LT_CHECK_LAUNCH();
    count_launches(1);
    int64_t nnz = 0;
    StatusBlock hst;
    LT_CUDA(cudaMemcpyAsync(&nnz, w.nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaMemcpyAsync(&hst, w.st, sizeof(StatusBlock), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    *nnz_out = nnz;
    if (hst.code != 0) return (ltsnet_status)hst.code;
    if (nnz > cap) return LTSNET_ERR_WORKSPACE;
    return LTSNET_OK;
}
