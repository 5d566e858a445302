// Host-side parts of the C ABI: defaults, status strings, the status poll and
// instrumentation (launch counter, per-kernel CUDA-event timing).
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace lt {
namespace {

std::atomic<int64_t> g_launches{0};

struct Probe {
    bool on = false;
    int32_t cap = 0;
    int32_t used = 0;
    std::vector<cudaEvent_t> ev;  // start/stop pairs
};
std::mutex g_probe_mu;
Probe g_probe[4];

const ltsnet_stage kDefaultStages[2] = {
    {250, 1.0f, 1.2f, 0.0f, 1.0f, 0.5f},
    {750, 1.0f, 0.01f, 0.6f, 1.0f, 0.8f},
};

}  // namespace

namespace {
thread_local int64_t t_launches = 0;  // this thread's share of g_launches
}  // namespace

void count_launches(int64_t k)
{
    g_launches.fetch_add(k, std::memory_order_relaxed);
    t_launches += k;
}

int64_t thread_launch_count() { return t_launches; }

namespace {
constexpr int kMaxDev = 64;
std::mutex g_dev_mu;
int g_sms[kMaxDev] = {};
bool g_once[kOnceSlots][kMaxDev] = {};
}  // namespace

int num_sms()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return kSplitBlocks;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_sms[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return kSplitBlocks;
        g_sms[dev] = v;
    }
    return g_sms[dev];
}

cudaError_t once_per_device(int slot, cudaError_t (*f)())
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev || slot < 0 || slot >= kOnceSlots) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_once[slot][dev]) return cudaSuccess;
    e = f();
    if (e == cudaSuccess) g_once[slot][dev] = true;
    return e;
}

namespace {
thread_local char g_err[256] = "";
}

void note_cuda_error(cudaError_t e, const char* where)
{
    snprintf(g_err, sizeof(g_err), "%s (%s) at %s", cudaGetErrorName(e), cudaGetErrorString(e), where);
}

bool profiling_active()
{
    std::lock_guard<std::mutex> lk(g_probe_mu);
    for (int k = 1; k <= 3; ++k)
        if (g_probe[k].on) return true;
    return false;
}

namespace {
// Per host thread and device: threads that drive different streams at once
// (ltsnet_run_batched) each capture and fork on their own streams.
struct AuxSet {
    AuxStreams a[64];
    ~AuxSet()
    {
        for (AuxStreams& x : a) {
            if (!x.ready) continue;
            cudaStreamDestroy(x.branch);
            cudaStreamDestroy(x.capture);
            cudaEventDestroy(x.fork);
            cudaEventDestroy(x.join);
        }
    }
};
thread_local AuxSet t_aux;
}  // namespace

// Internal non-blocking streams and events of the calling thread on the
// current device, created on first use (they carry the kernel-spectrum
// branch and graph capture).
cudaError_t aux_streams(AuxStreams** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    AuxStreams& a = t_aux.a[dev];
    if (!a.ready) {
        if ((e = cudaStreamCreateWithFlags(&a.branch, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&a.capture, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming)) != cudaSuccess) return e;
        a.ready = true;
    }
    *out = &a;
    return cudaSuccess;
}

void profile_start(int32_t kernel, cudaStream_t s)
{
    if (kernel < 1 || kernel > 3) return;
    std::lock_guard<std::mutex> lk(g_probe_mu);
    Probe& p = g_probe[kernel];
    if (!p.on || p.used >= p.cap) return;
    cudaEventRecord(p.ev[2 * p.used], s);
}

void profile_stop(int32_t kernel, cudaStream_t s)
{
    if (kernel < 1 || kernel > 3) return;
    std::lock_guard<std::mutex> lk(g_probe_mu);
    Probe& p = g_probe[kernel];
    if (!p.on || p.used >= p.cap) return;
    cudaEventRecord(p.ev[2 * p.used + 1], s);
    ++p.used;
}

}  // namespace lt

extern "C" ltsnet_params ltsnet_default_params(void)
{
    ltsnet_params p;
    p.perplexity = 30.0f;
    p.eps = 1.0f / 20.0f;
    p.nodes_per_box = 3;
    p.box_width_max = 0.25f;
    p.min_boxes = 50;
    p.max_boxes = 640;
    p.learning_rate = 0.0f;
    p.beta_max_steps = 100;
    p.beta_tol = 1e-5;
    p.n_stages = 2;
    p.stages = lt::kDefaultStages;
    p.flags = 0;
    p.conv_mode = LTSNET_CONV_FFT;
    return p;
}

extern "C" int32_t ltsnet_default_stages(int32_t total_iters, ltsnet_stage* out)
{
    if (!out || total_iters < 0) return 0;
    const int32_t first = total_iters < 250 ? total_iters : 250;
    out[0] = lt::kDefaultStages[0];
    out[0].iters = first;
    if (total_iters <= first) return 1;
    out[1] = lt::kDefaultStages[1];
    out[1].iters = total_iters - first;
    return 2;
}

extern "C" const char* ltsnet_status_string(ltsnet_status s)
{
    switch (s) {
        case LTSNET_OK: return "ok";
        case LTSNET_WARN_NOT_CONVERGED: return "warning: some rows did not reach the target perplexity";
        case LTSNET_ERR_INVALID_ARG: return "invalid argument";
        case LTSNET_ERR_WORKSPACE: return "workspace or output buffer too small (or misaligned)";
        case LTSNET_ERR_CUDA: return "CUDA runtime error";
        case LTSNET_ERR_DEVICE_TIMEOUT: return "a device loop reached its iteration cap";
        case LTSNET_ERR_NONFINITE: return "non-finite value in the layout or gradient";
        case LTSNET_ERR_BAD_GRAPH: return "graph column index out of range";
    }
    return "unknown status";
}

extern "C" ltsnet_status ltsnet_poll_status(void* ws, size_t ws_bytes, ltsnet_stream stream)
{
    if (!ws || ws_bytes < sizeof(lt::StatusBlock)) return LTSNET_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    lt::StatusBlock h;
    LT_CUDA(cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    LT_CUDA(cudaMemsetAsync(ws, 0, sizeof(h), s));
    LT_CUDA(cudaStreamSynchronize(s));
    if (h.code != 0) return (ltsnet_status)h.code;
    if (h.warn & 1) return LTSNET_WARN_NOT_CONVERGED;
    return LTSNET_OK;
}

extern "C" int64_t ltsnet_launch_count(void) { return lt::g_launches.load(); }

extern "C" const char* ltsnet_last_cuda_error(void) { return lt::g_err; }

extern "C" ltsnet_status ltsnet_profile_begin(int32_t kernel, int32_t max_launches)
{
    if (kernel < 1 || kernel > 3 || max_launches < 1) return LTSNET_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(lt::g_probe_mu);
    lt::Probe& p = lt::g_probe[kernel];
    for (cudaEvent_t e : p.ev) cudaEventDestroy(e);
    p.ev.assign(2 * (size_t)max_launches, nullptr);
    for (auto& e : p.ev) LT_CUDA(cudaEventCreate(&e));
    p.cap = max_launches;
    p.used = 0;
    p.on = true;
    return LTSNET_OK;
}

extern "C" ltsnet_status ltsnet_profile_end(int32_t kernel, double* total_ms, int32_t* launches)
{
    if (kernel < 1 || kernel > 3 || !total_ms || !launches) return LTSNET_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(lt::g_probe_mu);
    lt::Probe& p = lt::g_probe[kernel];
    double tot = 0.0;
    for (int32_t i = 0; i < p.used; ++i) {
        LT_CUDA(cudaEventSynchronize(p.ev[2 * i + 1]));
        float ms = 0.f;
        LT_CUDA(cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = p.used;
    for (cudaEvent_t e : p.ev) cudaEventDestroy(e);
    p.ev.clear();
    p.on = false;
    p.cap = p.used = 0;
    return LTSNET_OK;
}
