// Full single-source BFS, level-synchronous, for the Pivot MDS start and the
// stress metric.  One grid-wide launch expands one level: every frontier
// vertex claims its unreached neighbours (16-bit compare-and-swap on a
// uint16 distance row, 0xFFFF = unreached) and appends them to the other
// queue; the last block to finish swaps the queues.  The pivot or source,
// the queues and the counts live in a control block, so a batch of level
// launches is one CUDA graph replayed as often as the depth needs; the host
// checks the frontier once per batch.  No kernel waits on another.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace lt {
namespace {

constexpr int kBfsThreads = 256;
constexpr uint16_t kUnreached = 0xFFFF;
constexpr int kMaxDist = 65534;   // larger distances do not fit a uint16 row
constexpr int kLevelBatch = 64;   // level launches per graph replay

struct LevelCtl {
    int32_t row;      // distance row of the running BFS
    int32_t cur;      // queue holding the current frontier
    int32_t cnt[2];   // frontier sizes; cnt[cur ^ 1] is 0 between launches
    int32_t levels;   // frontiers expanded in the current BFS
    uint32_t ticket;  // blocks finished in the current launch
    int32_t err;      // 1: a distance above kMaxDist, 2: a column id out of range, 3: a bad source
    int32_t pad;
};

// Seeds row `row` of D with source `src` (the row must hold 0xFFFF).
__device__ __forceinline__ void bfs_seed(LevelCtl* ctl, uint16_t* D, int32_t n, int32_t row, int32_t src,
                                         int32_t* q0)
{
    ctl->row = row;
    ctl->cur = 0;
    ctl->cnt[1] = 0;
    ctl->levels = 0;
    ctl->ticket = 0;
    D[(size_t)row * n + src] = 0;
    q0[0] = src;
    ctl->cnt[0] = 1;
}

__global__ void __launch_bounds__(kBfsThreads) k_bfs_level(const int64_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col, int32_t n,
                                                           uint16_t* __restrict__ D, int32_t* __restrict__ q0,
                                                           int32_t* __restrict__ q1, LevelCtl* ctl, StatusBlock* st)
{
    const int cur = ctl->cur;
    const int32_t count = ctl->cnt[cur];
    if (count == 0) return;
    uint16_t* d = D + (size_t)ctl->row * n;
    const int32_t* qc = cur ? q1 : q0;
    int32_t* qn = cur ? q0 : q1;
    int32_t* ncnt = &ctl->cnt[cur ^ 1];
    const int lane = threadIdx.x & 31, grp = lane >> 3, sub = lane & 7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool overflow = false;
    // an 8-lane group per frontier vertex; every lane of the warp runs the
    // same number of trips so the ballot below sees the whole warp
    for (int64_t base = warp * 4; base < count; base += nwarps * 4) {
        const int64_t idx = base + grp;
        int64_t e0 = 0, e1 = 0;
        uint32_t lev = 0;
        if (idx < count) {
            const int32_t u = qc[idx];
            e0 = row_ptr[u];
            e1 = row_ptr[u + 1];
            lev = (uint32_t)d[u] + 1u;
        }
        int64_t trips = (e1 - e0 + 7) >> 3;
        trips = max(trips, (int64_t)__shfl_xor_sync(FULL, (long long)trips, 8));
        trips = max(trips, (int64_t)__shfl_xor_sync(FULL, (long long)trips, 16));
        for (int64_t r = 0; r < trips; ++r) {
            const int64_t e = e0 + r * 8 + sub;
            bool push = false;
            int32_t v = 0;
            if (e < e1) {
                v = col[e];
                if ((uint32_t)v >= (uint32_t)n) {
                    record_error(st, LTSNET_ERR_BAD_GRAPH, v);
                    ctl->err = 2;
                } else if (d[v] == kUnreached) {
                    if (lev > (uint32_t)kMaxDist) {
                        overflow = true;
                    } else {
                        push = atomicCAS(&d[v], kUnreached, (uint16_t)lev) == kUnreached;
                    }
                }
            }
            const unsigned b = __ballot_sync(FULL, push);
            if (b) {
                const int leader = __ffs(b) - 1;
                int32_t pos = 0;
                if (lane == leader) pos = atomicAdd(ncnt, __popc(b));
                pos = __shfl_sync(FULL, pos, leader);
                if (push) qn[pos + __popc(b & lanemask_lt())] = v;
            }
        }
    }
    if (overflow) {
        record_error(st, LTSNET_ERR_INVALID_ARG, kMaxDist);
        ctl->err = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&ctl->ticket, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            ctl->cnt[cur] = 0;
            ctl->cur = cur ^ 1;
            ctl->levels += 1;
            ctl->ticket = 0;
        }
    }
}

// Host: level launches for one graph, distance matrix and queue pair.
struct LevelRunner {
    const int64_t* row_ptr;
    const int32_t* col;
    int32_t n;
    uint16_t* D;
    int32_t* q0;
    int32_t* q1;
    LevelCtl* ctl;
    StatusBlock* st;
    cudaGraphExec_t exec = nullptr;
    int32_t reps = 1;  // graph replays before the first check of the next BFS
    unsigned grid = 2u * (unsigned)num_sms();  // two waves of blocks per SM

    ~LevelRunner()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }

    // Captures kLevelBatch launches on the library's capture stream (the
    // launches are issued directly when graphs are off, e.g. while kernels
    // are being timed one by one).
    ltsnet_status prepare()
    {
        AuxStreams* aux = nullptr;
        if (profiling_active() || aux_streams(&aux) != cudaSuccess) return LTSNET_OK;
        cudaGraph_t graph = nullptr;
        LT_CUDA(cudaStreamBeginCapture(aux->capture, cudaStreamCaptureModeThreadLocal));
        for (int b = 0; b < kLevelBatch; ++b)
            k_bfs_level<<<grid, kBfsThreads, 0, aux->capture>>>(row_ptr, col, n, D, q0, q1, ctl, st);
        cudaError_t e1 = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(aux->capture, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            LT_CUDA(e1 != cudaSuccess ? e1 : e2);
        }
        cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        LT_CUDA(e3);
        return LTSNET_OK;
    }

    // Runs the BFS seeded in the control block to its end (synchronous).
    // *h gets the final control block; h->err != 0 means the BFS stopped on
    // an error (the status word in `st` says which).
    ltsnet_status run(cudaStream_t s, LevelCtl* h)
    {
        int64_t launched = 0;
        for (;;) {
            // a BFS that has not ended after kMaxDist + 2 levels would have
            // set err; more launches than that mean a broken count
            if (launched > kMaxDist + 2 * kLevelBatch) return LTSNET_ERR_DEVICE_TIMEOUT;
            launched += (int64_t)reps * kLevelBatch;
            for (int32_t q = 0; q < reps; ++q) {
                if (exec) {
                    LT_CUDA(cudaGraphLaunch(exec, s));
                } else {
                    for (int b = 0; b < kLevelBatch; ++b)
                        k_bfs_level<<<grid, kBfsThreads, 0, s>>>(row_ptr, col, n, D, q0, q1, ctl, st);
                    LT_CHECK_LAUNCH();
                }
                count_launches(kLevelBatch);
            }
            LT_CUDA(cudaMemcpyAsync(h, ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, s));
            LT_CUDA(cudaStreamSynchronize(s));
            if (h->err || h->cnt[h->cur] == 0) break;
            reps = std::min<int32_t>(reps * 2, 64);
        }
        // the next BFS starts with enough batches for this one's depth
        reps = std::max<int32_t>(1, (h->levels + kLevelBatch) / kLevelBatch);
        return LTSNET_OK;
    }
};

}  // namespace
}  // namespace lt
