// Internal declarations shared by the translation units of libprofusion.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>

#include "../../include/profusion.h"

// --------------------------------------------------------------------------
// TSDF value encoding in the f32 tsdf array.
//
// A node is usable by the fitness when it is observed and within the
// truncation band (|tsdf| < 1).  Storing the other nodes as non-finite
// values makes that test fall out of the interpolation itself: a linear
// interpolation with a NaN or infinite end point is never finite, so the
// trilinear value of a cell is finite exactly when all eight nodes are
// usable.  Encoding:
//   unobserved (weight 0)        -> quiet NaN
//   observed, tsdf == +1 / -1    -> +inf / -inf
//   observed, |tsdf| < 1         -> the value
// --------------------------------------------------------------------------
#define PF_UNOBSERVED __int_as_float(0x7fc00000)

__host__ __device__ inline float pf_encode(float t, float w)
{
#ifdef __CUDA_ARCH__
    if (!(w > 0.0f)) return __int_as_float(0x7fc00000);
    if (t >= 1.0f) return __int_as_float(0x7f800000);
    if (t <= -1.0f) return __int_as_float(0xff800000);
    return t;
#else
    if (!(w > 0.0f)) return NAN;
    if (t >= 1.0f) return INFINITY;
    if (t <= -1.0f) return -INFINITY;
    return t;
#endif
}

// Value of an observed node (weight > 0): infinities stand for +-1.
__host__ __device__ inline float pf_decode(float e)
{
    return isinf(e) ? copysignf(1.0f, e) : e;
}

// --------------------------------------------------------------------------
// Storage types.  The tsdf (and the cell view) are stored as float, half,
// bfloat16 or scaled e4m3 -- the encoding above survives the conversion
// (NaN and infinities are kept; e4m3 codes them as below) and a value that
// rounds to +-1 is stored as +-infinity, so a finite stored value always
// lies inside the band -- and the weight as float or uint8.  All arithmetic
// is float.
// --------------------------------------------------------------------------
__host__ __device__ inline float pf_to_float(float v) { return v; }
__host__ __device__ inline float pf_to_float(__half v) { return __half2float(v); }
__host__ __device__ inline float pf_to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__host__ __device__ inline float pf_to_float(uint8_t v) { return (float)v; }

// 8-bit storage (PF_FP8E4M3): the value scaled by 2^8 in e4m3 (a value in
// (-1, 1) keeps 3 mantissa bits; the scale lifts the values near the surface
// out of the e4m3 subnormals).  e4m3 has no infinities: the largest finite
// code, +-448, stands for the outside-the-band +-1 and the NaN code for
// unobserved.  Scaled values stay below 256 in magnitude, so 448 never
// collides with a value.
constexpr float PF_FP8_SCALE = 256.0f;
constexpr unsigned char PF_FP8_NAN = 0x7f, PF_FP8_POS = 0x7e, PF_FP8_NEG = 0xfe;
__host__ __device__ inline float pf_to_float(__nv_fp8_e4m3 v)
{
    const __half h(__nv_cvt_fp8_to_halfraw(v.__x, __NV_E4M3));
    const float f = __half2float(h);
    if (f != f) return f;
    return fabsf(f) >= 448.0f ? copysignf(INFINITY, f) : f * (1.0f / PF_FP8_SCALE);
}

template <typename T> __host__ __device__ inline T pf_from_float(float v);
template <> __host__ __device__ inline float pf_from_float<float>(float v) { return v; }
template <> __host__ __device__ inline __half pf_from_float<__half>(float v)
{
    const float r = __half2float(__float2half_rn(v));
    return __float2half_rn(r >= 1.0f ? INFINITY : (r <= -1.0f ? -INFINITY : v));
}
template <> __host__ __device__ inline __nv_bfloat16 pf_from_float<__nv_bfloat16>(float v)
{
    const float r = __bfloat162float(__float2bfloat16_rn(v));
    return __float2bfloat16_rn(r >= 1.0f ? INFINITY : (r <= -1.0f ? -INFINITY : v));
}
template <> __host__ __device__ inline uint8_t pf_from_float<uint8_t>(float v) { return (uint8_t)v; }
template <> __host__ __device__ inline __nv_fp8_e4m3 pf_from_float<__nv_fp8_e4m3>(float v)
{
    __nv_fp8_e4m3 r;
    if (v != v) {
        r.__x = PF_FP8_NAN;
    } else if (v >= 1.0f || v <= -1.0f) {
        r.__x = v > 0.0f ? PF_FP8_POS : PF_FP8_NEG;
    } else {
        r.__x = __nv_cvt_float_to_fp8(v * PF_FP8_SCALE, __NV_SATFINITE, __NV_E4M3);
        const float back = __half2float(__half(__nv_cvt_fp8_to_halfraw(r.__x, __NV_E4M3)));
        if (back >= PF_FP8_SCALE) r.__x = PF_FP8_POS;       // rounds to +-1: outside the band
        else if (back <= -PF_FP8_SCALE) r.__x = PF_FP8_NEG;
    }
    return r;
}

inline size_t pf_dtype_size(pf_dtype t) { return t == PF_F32 ? 4 : t == PF_FP8E4M3 ? 1 : 2; }

// --------------------------------------------------------------------------
// Volume and workspace
// --------------------------------------------------------------------------
struct pf_workspace {
    int pix_cap = 0;        // max pixels per frame
    int k_cap = 0;          // max particles
    int part_cap = 0;       // partial slots (tiles x particles)
    float4* points = nullptr;        // pix_cap
    int* block_counts = nullptr;     // back-projection blocks
    int* n_points = nullptr;         // 1
    float* part_S = nullptr;         // part_cap
    int* part_C = nullptr;           // part_cap
    unsigned int* counter = nullptr; // last-block tickets (zeroed, reset by the last block)
    void* chunks = nullptr;          // the particle chunks of a search iteration, see track.cu
    int chunk_cap = 0;               // chunks it holds
    unsigned int* chunk_counter = nullptr;  // per chunk: tickets of its point tiles (zeroed, reset by the last)
    float* chunk_E = nullptr;        // per particle: fitness of the search iteration (chunk_cap x 32)
    int* chunk_C = nullptr;          // per particle: valid points
    // decimated point sets in a locality order (see track.cu): each point's
    // tile, the reordered kept points of up to three strides, counters
    int* point_tile = nullptr;       // pix_cap
    float4* kept = nullptr;          // 2 x pix_cap
    int* kept_count = nullptr;       // 3: kept points of each stride
    int* order_scratch = nullptr;    // order_cap: per (block of tiles, tile row) counts and first indices, offsets
    int order_cap = 0;
    double* state = nullptr;         // search state, see track.cu
    double* pose_in = nullptr;       // 16 (sync entry point)
    double* pose_out = nullptr;      // 16
    pf_track_stats* stats = nullptr; // 1
};

// Fusion works on tiles of 32 x 8 x 8 nodes; the cell view is refreshed
// tile by tile after fusion.
constexpr int PF_TX = 32, PF_TY = 8, PF_TZ = 8;

// Per-fusion tile lists (device memory, one slot per tile): the tiles that
// survive the frustum cull with the camera-frame position of their first
// node, and the tiles whose cell-view records must be rewritten.
struct FusionList {
    int* count = nullptr;         // [0] fused tiles, [1] tiles to refresh
    int* tile = nullptr;          // fused tile indices
    float4* base = nullptr;       // their first node in the camera frame: x, y, z hi, z lo
    float* step = nullptr;        // 9: camera-frame step per node index along i, j, k
    int* refresh_tile = nullptr;  // tiles to refresh
};

struct pf_volume {
    pf_volume_desc desc;
    int device = 0;
    size_t n_nodes = 0;
    void* tsdf = nullptr;      // encoded, see above; float, half or bfloat16 (desc.tsdf_dtype)
    void* weight = nullptr;    // float, or uint8 when desc.weight_u8
    void* cells = nullptr;     // cell view: 8 values per node (the cell whose lower corner it is)
    float* cells32 = nullptr;  // 16-/8-bit grids, full view: the same records as floats (x-differences formed)
    int* tile_stamp = nullptr; // per fusion tile: stamp of the last fusion that reached it
    int stamp = 0;             // fusions so far
    int tiles[3] = {0, 0, 0};
    int fitness_variant = 0;
    pf_status last_status = PF_OK;  // last failing status of a call on this volume
    FusionList list;
    pf_workspace ws;
};

// Storage type of the cell view's records: the node array's, or the search
// view type of a float grid (pf_volume_desc.search_dtype).
inline pf_dtype pf_view_dtype(const pf_volume* v)
{
    return v->desc.search_dtype != PF_F32 ? v->desc.search_dtype : v->desc.tsdf_dtype;
}

// Type the fitness kernel is instantiated on for a layout: the cell view's
// (layout 3) or the node array's (layouts 1 and 2).
inline pf_dtype pf_fitness_dtype(const pf_volume* v, int layout)
{
    return layout == 3 ? pf_view_dtype(v) : v->desc.tsdf_dtype;
}

// --------------------------------------------------------------------------
// Host helpers
// --------------------------------------------------------------------------
namespace pf {

extern std::atomic<unsigned long long> g_launches;
extern std::atomic<unsigned long long> g_allocs;

inline void count_launch(unsigned n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Every device allocation the library makes goes through these two, so that
// pf_alloc_count can tell a caller whether a call allocated.
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes)
{
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

template <typename T>
inline cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t s)
{
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
}

enum KernelClass { KC_FITNESS = 0, KC_FITNESS1, KC_INTEGRATE, KC_REFRESH, KC_BACKPROJECT, KC_RAYCAST, KC_COUNT };

// Event bracketing of launches (no-ops unless timing is enabled).
void timing_begin(KernelClass kc, cudaStream_t s);
void timing_end(KernelClass kc, cudaStream_t s);

pf_status check_intrinsics(const pf_intrinsics* intr);
pf_status workspace_reserve(pf_volume* vol, int max_pixels, int k_max);

// Records a failing status (anything but PF_OK and PF_ERR_TRACK_LOST, which
// describes the frame rather than the call) in the volume it concerns.
inline pf_status keep_status(const pf_volume* v, pf_status s)
{
    if (v && s != PF_OK && s != PF_ERR_TRACK_LOST) const_cast<pf_volume*>(v)->last_status = s;
    return s;
}

inline pf_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return PF_OK;
    if (e == cudaErrorMemoryAllocation) return PF_ERR_OOM;
    return PF_ERR_CUDA;
}

}  // namespace pf

#define PF_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return pf::cuda_status(e_); \
    } while (0)

#define PF_LAUNCHED()                                   \
    do {                                                \
        cudaError_t e_ = cudaGetLastError();            \
        if (e_ != cudaSuccess) return pf::cuda_status(e_); \
    } while (0)

// Camera parameters in the form the kernels use.
struct CamK {
    int width, height;
    float fx, fy, cx, cy, dmin, dmax;
};

inline CamK make_cam(const pf_intrinsics* in)
{
    CamK c;
    c.width = in->width;
    c.height = in->height;
    c.fx = in->fx;
    c.fy = in->fy;
    c.cx = in->cx;
    c.cy = in->cy;
    c.dmin = in->depth_min;
    c.dmax = in->depth_max;
    return c;
}

__device__ inline bool pf_depth_usable(float z, float dmin, float dmax)
{
    return isfinite(z) && z >= dmin && z <= dmax;
}
