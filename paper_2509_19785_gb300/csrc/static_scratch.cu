// Symmetrisation without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need
// this step: plug-ins and embedded hosts that are handed a fixed device-memory
// budget and forbid allocation, and latency-sensitive loops that must not pay
// for cudaMalloc's implicit device synchronisation.  For them,
// ltsnet_symmetrize_static keeps its
// scratch in a file-scope device array that exists for as long as the library
// is loaded, on every GPU that loads it, and forwards to ltsnet_symmetrize.
//
// The array holds one call's sort buffers for at most kStaticEntries emitted
// entries (2 n k <= 2^18, about 5.2 MB).  Every call uses the same array and
// leaves its contents behind; ltsnet_symmetrize clears the status word and the
// nnz counter it reads and writes everything else before reading it.  Calls
// whose GPU work overlaps (other streams, other host threads) race on it.
#include <mutex>

#include "common.cuh"

namespace lt {
namespace {

constexpr int64_t kStaticEntries = (int64_t)1 << 18;
// Workspace layout of ltsnet_symmetrize for 2 n k = kStaticEntries, always
// its compact form at these sizes (status, nnz, two 8-byte key buffers,
// histograms, scan temporaries), rounded up; checked against the exact size
// at every call.
constexpr size_t kStaticBytes = (size_t)kStaticEntries * 16 + ((size_t)1 << 20);

static __device__ __align__(256) unsigned char g_sym_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, resolved by the
// first call on each device (cudaGetSymbolAddress, which also loads the module
// there if needed); that first call should therefore come before any stream
// capture on the device.
ltsnet_status scratch_for_current_device(void** out)
{
    int dev = -1;
    LT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LTSNET_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        LT_CUDA(cudaGetSymbolAddress(&p, g_sym_scratch));
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return LTSNET_OK;
}

}  // namespace
}  // namespace lt

extern "C" int64_t ltsnet_symmetrize_static_max_entries(void) { return lt::kStaticEntries; }

extern "C" ltsnet_status ltsnet_symmetrize_static(const int32_t* nbr, const int32_t* cnt, const double* pcond,
                                                  int32_t n, int32_t k, int64_t* P_row, int32_t* P_col,
                                                  float* P_val, int64_t cap, int64_t* nnz_out,
                                                  ltsnet_stream stream)
{
    using namespace lt;
    if (n < 0 || k < 1) return LTSNET_ERR_INVALID_ARG;
    if (2 * (int64_t)n * k > kStaticEntries) return LTSNET_ERR_WORKSPACE;
    const size_t need = ltsnet_symmetrize_workspace_size(n, k);
    if (need > kStaticBytes) return LTSNET_ERR_WORKSPACE;
    void* ws = nullptr;
    const ltsnet_status rc = scratch_for_current_device(&ws);
    if (rc != LTSNET_OK) return rc;
    return ltsnet_symmetrize(nbr, cnt, pcond, n, k, P_row, P_col, P_val, cap, nnz_out, ws, kStaticBytes, stream);
}
