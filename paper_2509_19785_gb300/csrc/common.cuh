// Shared device/host helpers of the L-tsNET GB300 library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ltsnet.h"

namespace lt {

constexpr unsigned FULL = 0xffffffffu;
// Fixed block count of the kernels whose per-block partial sums live in the
// workspace or on the host stack: a constant, so that workspace sizes and the
// order of those sums do not depend on the device (152 = GB300's SM count).
constexpr int kSplitBlocks = 152;

// Status block at the start of every workspace (256 bytes).
struct StatusBlock {
    int32_t code;    // first error (ltsnet_status) recorded by a kernel, 0 if none
    int32_t detail;  // kernel-specific detail (e.g. the offending vertex)
    int32_t warn;    // LTSNET_WARN_* bits
    int32_t pad[61];
};
static_assert(sizeof(StatusBlock) == 256, "status block is 256 bytes");

__device__ __forceinline__ void record_error(StatusBlock* st, int32_t code, int32_t detail)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

// Order-preserving map float <-> int32 so that atomicMin/atomicMax on ints
// give the float min/max (negative floats have their magnitude bits flipped).
__device__ __forceinline__ int32_t f2ord(float f)
{
    int32_t i = __float_as_int(f);
    return i >= 0 ? i : (i ^ 0x7fffffff);
}
__device__ __forceinline__ float ord2f(int32_t i) { return __int_as_float(i >= 0 ? i : (i ^ 0x7fffffff)); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Host: SM count of the current device (queried once per device); launch
// sizes that should fill the GPU in waves take multiples of it.
int num_sms();
// Host: runs `f` once per (slot, device) and remembers success, so that a
// kernel's function attribute (which the runtime keeps per device) is raised
// on every device that launches it; thread-safe.  A failure is returned and
// retried on the next call.
enum OnceSlot { kOnceGridAttrs = 0, kOnceFusedAttrs, kOnceRadix, kOnceCalib, kOnceDft, kOnceSlots };
cudaError_t once_per_device(int slot, cudaError_t (*f)());
// Host: kernels launched by this library (instrumentation).
void count_launches(int64_t k);
// Launches counted by the calling thread (a capture on one thread measures
// its own graph's size while other threads launch).
int64_t thread_launch_count();
// Host: remember the last failing CUDA call of this thread (ltsnet_last_cuda_error).
void note_cuda_error(cudaError_t e, const char* where);
// Host: internal streams/events of a device (abi.cu).
struct AuxStreams {
    bool ready = false;
    cudaStream_t branch = nullptr, capture = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
cudaError_t aux_streams(AuxStreams** out);
bool profiling_active();
// Host: per-kernel event timing hooks (no-ops unless profiling is enabled).
void profile_start(int32_t kernel, cudaStream_t s);
void profile_stop(int32_t kernel, cudaStream_t s);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-provided workspace.
struct Carve {
    char* base;
    size_t cap;
    size_t off;
    Carve(void* b, size_t c) : base((char*)b), cap(c), off(0) {}
    template <typename T>
    T* take(size_t count)
    {
        off = align_up(off, 256);
        T* p = (T*)(base ? base + off : nullptr);
        off += sizeof(T) * count;
        return p;
    }
    bool ok() const { return off <= cap; }
};

}  // namespace lt

#define LT_STR2(x) #x
#define LT_STR(x) LT_STR2(x)

#define LT_CHECK_LAUNCH()                                              \
    do {                                                               \
        cudaError_t e_ = cudaGetLastError();                           \
        if (e_ != cudaSuccess) {                                       \
            ::lt::note_cuda_error(e_, __FILE__ ":" LT_STR(__LINE__));  \
            return LTSNET_ERR_CUDA;                                    \
        }                                                              \
    } while (0)

#define LT_CUDA(x)                                                     \
    do {                                                               \
        cudaError_t e_ = (x);                                          \
        if (e_ != cudaSuccess) {                                       \
            ::lt::note_cuda_error(e_, __FILE__ ":" LT_STR(__LINE__));  \
            return LTSNET_ERR_CUDA;                                    \
        }                                                              \
    } while (0)
