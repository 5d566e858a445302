// Vertex renumbering for locality (not a step of the method: the layout is
// the same up to floating-point summation order).
//
// The attraction pass gathers the coordinates of every P-neighbour of every
// vertex; with the input's own numbering those reads can be spread over the
// whole layout array.  Numbering the vertices in breadth-first discovery
// order (the Cuthill-McKee idea) puts graph neighbours -- and P's rows are
// graph balls -- at nearby indices, so the gathers hit the L1 cache.
//
// The order is exactly that of a sequential FIFO BFS that scans adjacency
// lists in stored order, restarted from the smallest unvisited vertex for
// each new component.  Level-synchronous on the GPU: for the frontier
// order[head, tail), every unvisited neighbour v takes the smallest key
// (frontier position, adjacency index) that reaches it (64-bit atomicMin);
// each frontier vertex then counts and places, in adjacency order, the
// neighbours whose key it holds, after an exclusive scan of those counts.
#include "common.cuh"

namespace lt {
namespace {

struct OrderCtl {
    int32_t head, tail;  // current frontier = order[head, tail)
    int32_t level;       // level of the current frontier
    int32_t total;       // children found for the next frontier
    int32_t cursor;      // no unvisited vertex below this id
    int32_t done;
    int32_t ticket;
    int32_t pad;
};

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int64_t kMaxOrderLevels = 4096;

__global__ void k_order_init(int32_t n, int32_t* __restrict__ level, unsigned long long* __restrict__ key,
                             int32_t* __restrict__ order, OrderCtl* ctl)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        level[v] = v == 0 ? 0 : -1;
        key[v] = ~0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        order[0] = 0;
        ctl->head = 0;
        ctl->tail = 1;
        ctl->level = 0;
        ctl->total = 0;
        ctl->cursor = 1;
        ctl->done = n <= 1;
        ctl->ticket = 0;
    }
}

// Every unvisited neighbour keeps the smallest (frontier position, index).
__global__ void k_order_expand(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int32_t n,
                               int32_t* __restrict__ level, unsigned long long* __restrict__ key,
                               const int32_t* __restrict__ order, const OrderCtl* __restrict__ ctl)
{
    if (ctl->done) return;
    const int lane = threadIdx.x & 31;
    const int32_t head = ctl->head, tail = ctl->tail, L = ctl->level;
    for (int64_t p = head + (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); p < tail;
         p += (int64_t)gridDim.x * kWarps) {
        const int32_t u = order[p];
        const int64_t a = row_ptr[u], b = row_ptr[u + 1];
        for (int64_t j = lane; j < b - a; j += 32) {
            const int32_t v = col[a + j];
            if ((unsigned)v >= (unsigned)n) continue;
            const int32_t lv = level[v];
            if (lv == -1 || lv == L + 1) {
                atomicMin(&key[v], ((unsigned long long)p << 32) | (unsigned long long)j);
                if (lv == -1) atomicCAS(&level[v], -1, L + 1);
            }
        }
    }
}

__device__ __forceinline__ bool is_child(const int32_t* __restrict__ level, const unsigned long long* __restrict__ key,
                                         int32_t v, int32_t n, int32_t L, int64_t p, int64_t j)
{
    return (unsigned)v < (unsigned)n && level[v] == L + 1 &&
           key[v] == (((unsigned long long)p << 32) | (unsigned long long)j);
}

__global__ void k_order_count(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int32_t n,
                              const int32_t* __restrict__ level, const unsigned long long* __restrict__ key,
                              const int32_t* __restrict__ order, int32_t* __restrict__ nchild,
                              const OrderCtl* __restrict__ ctl)
{
    if (ctl->done) return;
    const int lane = threadIdx.x & 31;
    const int32_t head = ctl->head, tail = ctl->tail, L = ctl->level;
    for (int64_t p = head + (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); p < tail;
         p += (int64_t)gridDim.x * kWarps) {
        const int32_t u = order[p];
        const int64_t a = row_ptr[u], b = row_ptr[u + 1];
        int c = 0;
        for (int64_t j = lane; j < b - a; j += 32) c += is_child(level, key, col[a + j], n, L, p, j) ? 1 : 0;
        c = warp_sum(c);
        if (lane == 0) nchild[p] = c;
    }
}

// Single block: exclusive scan of nchild over the frontier (into coff).
__global__ void __launch_bounds__(1024) k_order_scan(const int32_t* __restrict__ nchild, int32_t* __restrict__ coff,
                                                     OrderCtl* ctl)
{
    if (ctl->done) return;
    __shared__ int32_t wsum[33];
    __shared__ int32_t carry;
    const int32_t head = ctl->head, tail = ctl->tail;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t p0 = head; p0 < tail; p0 += blockDim.x) {
        const int64_t p = p0 + threadIdx.x;
        const int v = p < tail ? nchild[p] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        if (w == 0) {
            const int x = lane < nw ? wsum[lane] : 0;
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, xi, o);
                if (lane >= o) xi += t;
            }
            if (lane < nw) wsum[lane] = xi - x;
            if (lane == 31) wsum[32] = xi;
        }
        __syncthreads();
        if (p < tail) coff[p] = carry + wsum[w] + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) ctl->total = carry;
}

// Place the children in adjacency order; the last block advances the
// frontier, or starts the next component from the smallest unvisited vertex.
__global__ void k_order_place(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int32_t n,
                              int32_t* __restrict__ level, const unsigned long long* __restrict__ key,
                              int32_t* __restrict__ order, const int32_t* __restrict__ coff, OrderCtl* ctl)
{
    if (ctl->done) return;
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
    const unsigned ltm = lanemask_lt();
    const int32_t head = ctl->head, tail = ctl->tail, L = ctl->level;
    for (int64_t p = head + (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); p < tail;
         p += (int64_t)gridDim.x * kWarps) {
        const int32_t u = order[p];
        const int64_t a = row_ptr[u], b = row_ptr[u + 1];
        int64_t base = (int64_t)tail + coff[p];
        for (int64_t j0 = 0; j0 < b - a; j0 += 32) {
            const int64_t j = j0 + lane;
            const int32_t v = j < b - a ? col[a + j] : -1;
            const bool c = j < b - a && is_child(level, key, v, n, L, p, j);
            const unsigned bal = __ballot_sync(FULL, c);
            if (c) order[base + __popc(bal & ltm)] = v;
            base += __popc(bal);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ int32_t need_root, found;
    if (threadIdx.x == 0) {
        const int32_t total = ((volatile OrderCtl*)ctl)->total;
        ctl->ticket = 0;
        ctl->head = tail;
        ctl->tail = tail + total;
        ctl->level = L + 1;
        need_root = (total == 0 && tail < n) ? 1 : 0;
        if (tail + total >= n) ctl->done = 1;
    }
    __syncthreads();
    if (!need_root) return;
    // frontier exhausted with vertices left: smallest unvisited id from the cursor
    for (int32_t c0 = ((volatile OrderCtl*)ctl)->cursor; c0 < n; c0 += blockDim.x) {
        if (threadIdx.x == 0) found = 0x7fffffff;
        __syncthreads();
        const int32_t v = c0 + threadIdx.x;
        if (v < n && ((volatile int32_t*)level)[v] == -1) atomicMin(&found, v);
        __syncthreads();
        if (found != 0x7fffffff) break;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (found != 0x7fffffff) {
            level[found] = L + 1;
            order[tail] = found;
            ctl->tail = tail + 1;
            ctl->cursor = found + 1;
        } else {
            ctl->done = 1;  // cannot happen: tail < n leaves an unvisited vertex
        }
    }
}

__global__ void k_permute_rows(const int32_t* __restrict__ order, const int32_t* __restrict__ inv,
                               const int32_t* __restrict__ nbr, const double* __restrict__ pcond,
                               const int32_t* __restrict__ cnt, int32_t n, int32_t k, int32_t* __restrict__ nbr2,
                               double* __restrict__ pcond2, int32_t* __restrict__ cnt2)
{
    const int64_t nk = (int64_t)n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int s = (int)(e - i * k);
        const int32_t src = order[i];
        const int32_t v = nbr[(int64_t)src * k + s];
        nbr2[e] = (unsigned)v < (unsigned)n ? inv[v] : -1;
        pcond2[e] = pcond[(int64_t)src * k + s];
        if (s == 0) cnt2[i] = cnt[src];
    }
}

__global__ void k_inverse(const int32_t* __restrict__ order, int32_t n, int32_t* __restrict__ inv)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        inv[order[i]] = (int32_t)i;
}

__global__ void k_gather_rows2(const float2* __restrict__ src, const int32_t* __restrict__ idx, int32_t n,
                               float2* __restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

}  // namespace

size_t order_ws_bytes(int32_t n)
{
    Carve c(nullptr, 0);
    c.take<OrderCtl>(1);
    c.take<int32_t>(n);               // level
    c.take<unsigned long long>(n);    // key
    c.take<int32_t>(n);               // nchild
    c.take<int32_t>(n);               // coff
    return align_up(c.off, 256);
}

// Breadth-first order: order[new] = old, inv[old] = new.
cudaError_t bfs_order(const int64_t* row_ptr, const int32_t* col, int32_t n, int32_t* order, int32_t* inv, void* ws,
                      cudaStream_t s, bool* reordered)
{
    Carve c(ws, order_ws_bytes(n));
    OrderCtl* ctl = c.take<OrderCtl>(1);
    int32_t* level = c.take<int32_t>(n);
    unsigned long long* key = c.take<unsigned long long>(n);
    int32_t* nchild = c.take<int32_t>(n);
    int32_t* coff = c.take<int32_t>(n);
    const unsigned grid = num_sms() * 4;
    k_order_init<<<grid, kThreads, 0, s>>>(n, level, key, order, ctl);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Levels are launched in batches; a batch after the last level does
    // nothing (every kernel checks the done flag).  Graphs with more than
    // kMaxOrderLevels levels (long paths) are left in their own order:
    // *reordered = false, and the caller keeps the identity.
    const int batch = 16;
    int32_t done = 0;
    *reordered = false;
    for (int64_t lv = 0; lv < kMaxOrderLevels && !done; lv += batch) {
        for (int b = 0; b < batch; ++b) {
            k_order_expand<<<grid, kThreads, 0, s>>>(row_ptr, col, n, level, key, order, ctl);
            k_order_count<<<grid, kThreads, 0, s>>>(row_ptr, col, n, level, key, order, nchild, ctl);
            k_order_scan<<<1, 1024, 0, s>>>(nchild, coff, ctl);
            k_order_place<<<grid, kThreads, 0, s>>>(row_ptr, col, n, level, key, order, coff, ctl);
            count_launches(4);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&done, &ctl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    }
    if (!done) return cudaSuccess;
    k_inverse<<<grid, kThreads, 0, s>>>(order, n, inv);
    count_launches(1);
    *reordered = true;
    return cudaGetLastError();
}

cudaError_t permute_conditional_rows(const int32_t* order, const int32_t* inv, const int32_t* nbr,
                                     const double* pcond, const int32_t* cnt, int32_t n, int32_t k, int32_t* nbr2,
                                     double* pcond2, int32_t* cnt2, cudaStream_t s)
{
    k_permute_rows<<<num_sms() * 8, kThreads, 0, s>>>(order, inv, nbr, pcond, cnt, n, k, nbr2, pcond2, cnt2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t gather_rows2(const float2* src, const int32_t* idx, int32_t n, float2* dst, cudaStream_t s)
{
    k_gather_rows2<<<num_sms() * 4, kThreads, 0, s>>>(src, idx, n, dst);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lt

extern "C" size_t ltsnet_bfs_order_workspace_size(int32_t n)
{
    if (n < 0) return 0;
    return lt::order_ws_bytes(n);
}

extern "C" ltsnet_status ltsnet_bfs_order(const int64_t* row_ptr, const int32_t* col, int32_t n, int32_t* order,
                                          int32_t* inv, int32_t* reordered, void* ws, size_t ws_bytes,
                                          ltsnet_stream stream)
{
    using namespace lt;
    if (n < 1 || !row_ptr || !col || !order || !inv || !reordered || !ws) return LTSNET_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255) || ws_bytes < order_ws_bytes(n)) return LTSNET_ERR_WORKSPACE;
    bool r = false;
    LT_CUDA(bfs_order(row_ptr, col, n, order, inv, ws, (cudaStream_t)stream, &r));
    LT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    *reordered = r ? 1 : 0;
    return LTSNET_OK;
}
