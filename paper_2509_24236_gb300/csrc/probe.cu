// Instrumentation: the memory ceilings the fitness kernel is measured against.
//
// The fitness kernel (Sec. III-B, the fitness E) reads one 32-byte cell
// record per sample -- the eight corner values of the cell the transformed
// point falls in -- from the band of the grid around the observed surface.
// On the 640x480 / 512^3 workload that band (tens of MB) stays in the 129 MB
// L2, so the bytes a sample needs come from L2 (and L1), not from HBM.  This
// probe measures the two ceilings for such reads on the device it runs on:
//   mode 0  L2 -> SM bandwidth: every warp reads 32 consecutive records
//           (1 KiB) at a random 1 KiB-aligned position, bypassing L1
//           (ld.global.cg), so each byte crosses from L2 once and the L1
//           data pipe is not the limit;
//   mode 1  scattered records: every lane reads one record at a random
//           position with the load the fitness kernel uses
//           (ld.global.nc.v8.f32), the ceiling of a gather in which no two
//           lanes share a sector.
// Positions come from a per-warp (mode 0) or per-lane (mode 1) linear
// congruential sequence; each thread writes the sum of the values it loaded,
// so no load can be dropped, and a test can recompute that sum.
#include "pf_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 4;

__device__ __forceinline__ unsigned probe_next(unsigned h) { return h * 1664525u + 1013904223u; }

__device__ __forceinline__ unsigned probe_seed(unsigned x)
{
    // one round of a 32-bit integer mix (murmur3's finaliser), so that
    // neighbouring threads start far apart in the sequence
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

template <int MODE>
__global__ void __launch_bounds__(PROBE_THREADS) gather_probe_kernel(const float* __restrict__ buf,
                                                                      unsigned n_records, int loads, float* out)
{
    const unsigned tid = blockIdx.x * PROBE_THREADS + threadIdx.x;
    const unsigned lane = threadIdx.x & 31;
    unsigned h = probe_seed(MODE == 0 ? (tid >> 5) : tid);
    const unsigned n_blocks = n_records >> 5;  // 1 KiB blocks (mode 0)
    float acc = 0.0f;
    for (int i = 0; i < loads; ++i) {
        h = probe_next(h);
        const unsigned rec = MODE == 0 ? (__umulhi(h, n_blocks) << 5) + lane : __umulhi(h, n_records);
        const float* p = buf + 8 * (size_t)rec;
        float v0, v1, v2, v3, v4, v5, v6, v7;
        if (MODE == 0)
            asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=f"(v0), "=f"(v1), "=f"(v2), "=f"(v3), "=f"(v4), "=f"(v5), "=f"(v6), "=f"(v7)
                         : "l"(p));
        else
            asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=f"(v0), "=f"(v1), "=f"(v2), "=f"(v3), "=f"(v4), "=f"(v5), "=f"(v6), "=f"(v7)
                         : "l"(p));
        acc += ((v0 + v1) + (v2 + v3)) + ((v4 + v5) + (v6 + v7));
    }
    out[tid] = acc;
}

}  // namespace

extern "C" pf_status pf_gather_probe(const float* buf_dev, long long n_records, int mode, int loads_per_thread,
                                     float* out_dev, long long* threads_out, void* stream)
{
    if (!threads_out) return PF_ERR_INVALID_ARG;
    if (mode < 0 || mode > 1 || loads_per_thread < 1) return PF_ERR_INVALID_ARG;
    if (n_records < 32 || n_records > (1ll << 31) || (n_records & 31)) return PF_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(buf_dev) & 31) return PF_ERR_INVALID_ARG;  // 32-byte records
    int dev = 0, sms = 0;
    PF_CUDA(cudaGetDevice(&dev));
    PF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * PROBE_CTAS_PER_SM;
    *threads_out = (long long)blocks * PROBE_THREADS;
    if (!out_dev) return PF_OK;  // a query of the output size
    if (!buf_dev) return PF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == 0)
        gather_probe_kernel<0><<<blocks, PROBE_THREADS, 0, s>>>(buf_dev, (unsigned)n_records, loads_per_thread,
                                                                out_dev);
    else
        gather_probe_kernel<1><<<blocks, PROBE_THREADS, 0, s>>>(buf_dev, (unsigned)n_records, loads_per_thread,
                                                                out_dev);
    pf::count_launch();
    PF_LAUNCHED();
    return PF_OK;
}
