// Status strings, argument checks shared by the entry points, launch
// accounting and the optional per-kernel-class event timing.
#include <mutex>
#include <string.h>
#include <vector>

#include "pf_internal.cuh"

namespace pf {

std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_allocs{0};

namespace {

struct EventPair {
    cudaEvent_t start, stop;
};

struct TimingState {
    std::mutex mu;
    bool enabled = false;
    std::vector<EventPair> pending[KC_COUNT];
    std::vector<EventPair> pool;
    EventPair open[KC_COUNT];
    bool is_open[KC_COUNT] = {};
};

TimingState& timing()
{
    static TimingState t;
    return t;
}

const char* kClassNames[KC_COUNT] = {"fitness", "fitness1", "integrate", "refresh", "backproject", "raycast"};

}  // namespace

void timing_begin(KernelClass kc, cudaStream_t s)
{
    TimingState& t = timing();
    std::lock_guard<std::mutex> lock(t.mu);
    if (!t.enabled) return;
    EventPair p;
    if (!t.pool.empty()) {
        p = t.pool.back();
        t.pool.pop_back();
    } else {
        if (cudaEventCreate(&p.start) != cudaSuccess) return;
        if (cudaEventCreate(&p.stop) != cudaSuccess) {
            cudaEventDestroy(p.start);
            return;
        }
    }
    cudaEventRecord(p.start, s);
    t.open[kc] = p;
    t.is_open[kc] = true;
}

void timing_end(KernelClass kc, cudaStream_t s)
{
    TimingState& t = timing();
    std::lock_guard<std::mutex> lock(t.mu);
    if (!t.enabled || !t.is_open[kc]) return;
    cudaEventRecord(t.open[kc].stop, s);
    t.pending[kc].push_back(t.open[kc]);
    t.is_open[kc] = false;
}

// Sets whether launches are timed; returns the previous setting (used to
// keep event records out of captured graphs).
bool timing_swap(bool enabled)
{
    TimingState& t = timing();
    std::lock_guard<std::mutex> lock(t.mu);
    const bool was = t.enabled;
    t.enabled = enabled;
    return was;
}

pf_status check_intrinsics(const pf_intrinsics* in)
{
    if (!in) return PF_ERR_INVALID_ARG;
    if (in->width < 1 || in->height < 1 || in->width > 16384 || in->height > 16384) return PF_ERR_INVALID_ARG;
    if (!(in->fx > 0.0f) || !(in->fy > 0.0f) || !std::isfinite(in->cx) || !std::isfinite(in->cy))
        return PF_ERR_INVALID_ARG;
    if (!(in->depth_min > 0.0f) || !(in->depth_max >= in->depth_min) || !std::isfinite(in->depth_max))
        return PF_ERR_INVALID_ARG;
    return PF_OK;
}

}  // namespace pf

extern "C" {

const char* pf_status_string(pf_status s)
{
    switch (s) {
    case PF_OK: return "ok";
    case PF_ERR_INVALID_ARG: return "invalid argument";
    case PF_ERR_OOM: return "out of device memory";
    case PF_ERR_CUDA: return "CUDA error";
    case PF_ERR_TIMEOUT: return "timed out";
    case PF_ERR_TRACK_LOST: return "tracking lost";
    case PF_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

unsigned long long pf_launch_count(void) { return pf::g_launches.load(); }

unsigned long long pf_alloc_count(void) { return pf::g_allocs.load(); }

pf_status pf_set_kernel_timing(int enable)
{
    pf::TimingState& t = pf::timing();
    std::lock_guard<std::mutex> lock(t.mu);
    t.enabled = enable != 0;
    return PF_OK;
}

pf_status pf_kernel_timing(const char* kernel_class, double* total_ms, long long* launches)
{
    if (!kernel_class || !total_ms || !launches) return PF_ERR_INVALID_ARG;
    int kc = -1;
    for (int i = 0; i < pf::KC_COUNT; ++i)
        if (strcmp(kernel_class, pf::kClassNames[i]) == 0) kc = i;
    if (kc < 0) return PF_ERR_INVALID_ARG;
    pf::TimingState& t = pf::timing();
    std::lock_guard<std::mutex> lock(t.mu);
    double total = 0.0;
    long long n = 0;
    pf_status st = PF_OK;
    for (auto& p : t.pending[kc]) {
        if (cudaEventSynchronize(p.stop) != cudaSuccess) {
            st = PF_ERR_CUDA;
            continue;
        }
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            total += ms;
            ++n;
        }
        t.pool.push_back(p);
    }
    t.pending[kc].clear();
    *total_ms = total;
    *launches = n;
    return st;
}

}  // extern "C"
