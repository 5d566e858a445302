// K1 -- partial BFS k-nearest neighbours (Sec. 3.1 "partial BFS", Alg. 3 C0).
//
// One warp per source vertex s.  The warp keeps the BFS queue (the source plus
// the vertices discovered so far, in discovery order) and a hash set of the
// visited vertices in shared memory.  Each step takes the next 32 adjacency
// entries of the queue -- the remaining entries of the head vertex followed by
// those of the vertices behind it -- so short adjacency lists are batched and
// long ones are streamed 32 at a time.  Within a step the lanes hold the
// entries in queue order; a lane's vertex is new if it is not in the visited
// set and no lower lane holds the same vertex, and new vertices take queue
// positions by a ballot prefix count.  This reproduces exactly the order of a
// sequential FIFO BFS that marks vertices when they are enqueued, including
// the early stop the moment k vertices other than s have been found.
#include "common.cuh"

namespace lt {
namespace {

__device__ __forceinline__ unsigned hslot(int32_t v, int hlog2)
{
    return ((unsigned)v * 0x9E3779B1u) >> (32 - hlog2);
}

__device__ __forceinline__ bool hash_contains(const int32_t* H, int hlog2, int32_t v)
{
    const unsigned mask = (1u << hlog2) - 1u;
    unsigned pos = hslot(v, hlog2);
    // The table holds at most k+1 keys in >= 2(k+1) slots, so an empty slot
    // always ends the probe.
    while (true) {
        int32_t x = H[pos];
        if (x == v) return true;
        if (x == -1) return false;
        pos = (pos + 1u) & mask;
    }
}

__device__ __forceinline__ void hash_insert(int32_t* H, int hlog2, int32_t v)
{
    const unsigned mask = (1u << hlog2) - 1u;
    unsigned pos = hslot(v, hlog2);
    while (atomicCAS(&H[pos], -1, v) != -1) pos = (pos + 1u) & mask;
}

__global__ void k_partial_bfs(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              int32_t n, int32_t k, int32_t hlog2, int32_t warp_bytes,
                              int32_t* __restrict__ nbr, uint16_t* __restrict__ hop,
                              int32_t* __restrict__ cnt, StatusBlock* st)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    unsigned char* base = smem + (size_t)wib * warp_bytes;
    int64_t* qstart = (int64_t*)base;                 // adjacency start of queue entry
    int32_t* hash = (int32_t*)(qstart + (k + 1));     // visited set
    const int hcap = 1 << hlog2;
    int32_t* qv = hash + hcap;                        // queue vertex
    int32_t* qdeg = qv + (k + 1);                     // queue vertex degree
    uint16_t* qhop = (uint16_t*)(qdeg + (k + 1));     // queue vertex hop distance
    const unsigned ltm = lanemask_lt();

    for (int64_t s = (int64_t)blockIdx.x * wpb + wib; s < n; s += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < hcap; i += 32) hash[i] = -1;
        __syncwarp();
        if (lane == 0) {
            hash[hslot((int32_t)s, hlog2)] = (int32_t)s;
            int64_t a = row_ptr[s], b = row_ptr[s + 1];
            qv[0] = (int32_t)s;
            qhop[0] = 0;
            qstart[0] = a;
            qdeg[0] = (int32_t)(b - a);
        }
        __syncwarp();
        int32_t* out_n = nbr + s * (int64_t)k;
        uint16_t* out_h = hop + s * (int64_t)k;
        int head = 0, off = 0, tail = 1, found = 0;
        while (found < k && head < tail) {
            // Remaining adjacency of queue entries head+lane (clamped at 32:
            // only the first 32 positions of the step matter).
            const int e = head + lane;
            int rem = 0;
            if (e < tail) rem = qdeg[e] - (lane == 0 ? off : 0);
            const int remc = rem < 32 ? rem : 32;
            int cum = remc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(FULL, cum, o);
                if (lane >= o) cum += t;
            }
            const int total = __shfl_sync(FULL, cum, 31);
            const int T = total < 32 ? total : 32;
            // Queue entry holding step position p = lane: number of entries
            // whose inclusive prefix is <= p (prefixes are non-decreasing).
            const int p = lane;
            int ei = 0;
#pragma unroll
            for (int b = 16; b >= 1; b >>= 1) {
                int c = __shfl_sync(FULL, cum, ei + b - 1);
                if (c <= p) ei += b;
            }
            const int prevc = __shfl_sync(FULL, cum, ei > 0 ? ei - 1 : 0);
            const int excl = ei > 0 ? prevc : 0;
            bool valid = p < T;
            int32_t v = -1;
            uint16_t hv = 0;
            if (valid) {
                const int q = head + ei;
                const int64_t a = qstart[q] + (ei == 0 ? off : 0) + (p - excl);
                v = col[a];
                hv = (uint16_t)(qhop[q] + 1);
                if ((unsigned)v >= (unsigned)n) {
                    record_error(st, LTSNET_ERR_BAD_GRAPH, v);
                    valid = false;
                    v = -1;
                }
            }
            // Advance the cursor by T positions.  Fully consumed entries are a
            // prefix of the lanes.
            const bool full = (e < tail) && (cum <= T) && (rem <= 32);
            const unsigned fb = __ballot_sync(FULL, full);
            const int nfull = __ffs(~fb) - 1 < 0 ? 32 : __ffs(~fb) - 1;
            const int cprev = __shfl_sync(FULL, cum, nfull > 0 ? nfull - 1 : 0);
            // Duplicates within the step: the lowest lane is the discovery.
            const unsigned peers = __match_any_sync(FULL, v);
            bool isnew = false;
            if (valid && (peers & ltm) == 0) isnew = !hash_contains(hash, hlog2, v);
            const unsigned nb = __ballot_sync(FULL, isnew);
            const int room = k - found;
            const int rank = __popc(nb & ltm);
            if (isnew && rank < room) {
                hash_insert(hash, hlog2, v);
                const int qi = tail + rank;
                const int64_t a = row_ptr[v], b = row_ptr[v + 1];
                qv[qi] = v;
                qhop[qi] = hv;
                qstart[qi] = a;
                qdeg[qi] = (int32_t)(b - a);
                out_n[found + rank] = v;
                out_h[found + rank] = hv;
            }
            const int nnew = __popc(nb);
            const int add = nnew < room ? nnew : room;
            if (nfull == 0) {
                off += T;
            } else {
                off = T - cprev;
                head += nfull;
            }
            found += add;
            tail += add;
            __syncwarp();
        }
        for (int j = found + lane; j < k; j += 32) {
            out_n[j] = -1;
            out_h[j] = 0;
        }
        if (lane == 0) cnt[s] = found;
        __syncwarp();
    }
}

}  // namespace

size_t bfs_warp_bytes(int k, int* hlog2_out)
{
    int hlog2 = 5;
    while ((1 << hlog2) < 2 * (k + 1)) ++hlog2;
    if (hlog2_out) *hlog2_out = hlog2;
    size_t b = 8 * (size_t)(k + 1) + 4 * ((size_t)1 << hlog2) + 4 * (size_t)(k + 1) * 2 + 2 * (size_t)(k + 1);
    return align_up(b, 16);
}

}  // namespace lt

extern "C" ltsnet_status ltsnet_knn_bfs(const int64_t* row_ptr, const int32_t* col, int32_t n, int32_t k,
                                        int32_t* nbr, uint16_t* hop, int32_t* cnt, void* ws,
                                        size_t ws_bytes, ltsnet_stream stream)
{
    using namespace lt;
    if (n < 0 || k < 1 || k > LTSNET_MAX_K) return LTSNET_ERR_INVALID_ARG;
    if (n == 0) return LTSNET_OK;
    if (!row_ptr || !col || !nbr || !hop || !cnt || !ws) return LTSNET_ERR_INVALID_ARG;
    if (ws_bytes < sizeof(StatusBlock) || ((uintptr_t)ws & 255)) return LTSNET_ERR_WORKSPACE;
    int hlog2 = 0;
    const size_t wb = bfs_warp_bytes(k, &hlog2);
    const size_t smem_cap = 200 * 1024;
    int wpb = (int)(smem_cap / wb);
    if (wpb > 8) wpb = 8;
    if (wpb < 1) return LTSNET_ERR_INVALID_ARG;
    const size_t smem = wb * wpb;
    cudaStream_t s = (cudaStream_t)stream;
    LT_CUDA(cudaFuncSetAttribute(k_partial_bfs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_partial_bfs, wpb * 32, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t want = ((int64_t)n + wpb - 1) / wpb;
    int64_t grid = (int64_t)num_sms() * per_sm;
    if (grid > want) grid = want;
    k_partial_bfs<<<(unsigned)grid, wpb * 32, smem, s>>>(row_ptr, col, n, k, hlog2, (int32_t)wb, nbr, hop, cnt,
                                                          (StatusBlock*)ws);
    LT_CHECK_LAUNCH();
    count_launches(1);
    return LTSNET_OK;
}
