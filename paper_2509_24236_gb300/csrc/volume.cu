// Volume lifetime, host transfer and projective TSDF fusion.
//
// Fusion follows the KinectFusion rule the paper adopts (Sec. III, "Method
// overview"): each node is transformed into the camera, projected to its
// nearest pixel, and, when that pixel has a usable depth d and the node lies
// no deeper than one truncation behind it, the truncated z-distance
// t = min(1, (d - z_c) / tau) enters a running average with weight 1.
//
// GB300 layout: one CTA per 32 x 8 x 8 tile of nodes (x fastest, so a warp
// touches one 128-byte line of each array per slice); the tile is dropped
// before any memory access when its bounding sphere lies outside the view
// frustum or beyond depth_max + tau.  Node loads and stores happen only for
// nodes that pass every test, so HBM traffic is proportional to the nodes
// actually updated.  The camera-frame depth of a node is formed as a
// double-precision tile base (split into a float pair) plus a small float
// offset, which keeps the signed distance accurate to ~1e-7 m at any
// distance from the grid origin.
#include <stdlib.h>
#include <string.h>

#include <cstring>
#include <vector>

#include <type_traits>

#include "pf_internal.cuh"

namespace pf {
void align_release(const pf_volume* v);  // align.cu
}

namespace {

constexpr int TX = PF_TX, TY = PF_TY, TZ = PF_TZ;

struct IntegArgs {
    void* tsdf;
    void* weight;
    int nx, ny, nz;
    float trunc;
    float max_weight;
    CamK cam;
    const float* depth;
    const double* pose_dev;             // camera-to-world pose in device memory, or null: use pose
    double pose[12];                    // row-major 3x4
    double origin[3];
    double vs;
    float plane[4][3];                  // inward normals of the four side planes of the frustum
    float zfar;                         // nodes deeper than this are never updated
    float radius;                       // bounding radius of a tile (+ margin)
    int* tile_stamp;                    // tiles with a changed node value get *stamp_dev (null: no cell view)
    const int* stamp_dev;               // fusion counter on the device
    int tiles[3];                       // fusion tiles per axis
    FusionList list;                    // tiles that survive the cull, with their bases
};

// Starts a fusion: empties the tile lists and, with a cell view, advances the
// fusion counter the tile stamps refer to (on the device, so a captured and
// replayed launch sequence still marks each fusion apart).
__global__ void fusion_begin_kernel(FusionList list, int* stamp_counter)
{
    if (threadIdx.x == 0) {
        list.count[0] = 0;
        list.count[1] = 0;
        if (stamp_counter) *stamp_counter += 1;
    }
}

// One thread per fusion tile of TX x TY x TZ nodes: the camera-frame
// position of the tile's first node, X_c = R^T (X_w - t) with
// X_w = origin + vs (i0, j0, k0), in FP64 -- kept as floats, the depth as a
// hi + lo pair -- and the frustum cull of the tile's bounding sphere.  A tile
// that survives is appended to the list (its position in the list depends on
// scheduling; each tile's nodes are fused once whatever the order, so the
// result does not).  Thread 0 also writes the per-index steps, vs times the
// rows of R, which every tile shares.
__global__ void __launch_bounds__(256) fusion_tiles_kernel(IntegArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_tiles = a.tiles[0] * a.tiles[1] * a.tiles[2];
    if (t >= n_tiles) return;
    const int bx = t % a.tiles[0], by = (t / a.tiles[0]) % a.tiles[1], bz = t / (a.tiles[0] * a.tiles[1]);
    const int i0 = bx * TX, j0 = by * TY, k0 = bz * TZ;
    const double* P = a.pose_dev ? a.pose_dev : a.pose;
    double Pl[12];
    for (int q = 0; q < 12; ++q) Pl[q] = P[q];
    const double Xw[3] = {a.origin[0] + a.vs * i0, a.origin[1] + a.vs * j0, a.origin[2] + a.vs * k0};
    const double d[3] = {Xw[0] - Pl[3], Xw[1] - Pl[7], Xw[2] - Pl[11]};
    double b[3], c[3], st[9];
    for (int r = 0; r < 3; ++r) {
        b[r] = Pl[r] * d[0] + Pl[4 + r] * d[1] + Pl[8 + r] * d[2];
        st[r] = a.vs * Pl[r];          // step along i
        st[3 + r] = a.vs * Pl[4 + r];  // step along j
        st[6 + r] = a.vs * Pl[8 + r];  // step along k
        c[r] = b[r] + 0.5 * (TX - 1) * st[r] + 0.5 * (TY - 1) * st[3 + r] + 0.5 * (TZ - 1) * st[6 + r];
    }
    if (t == 0)
        for (int q = 0; q < 9; ++q) a.list.step[q] = (float)st[q];
    const float cx = (float)c[0], cy = (float)c[1], cz = (float)c[2];
    bool skip = (cz + a.radius <= 0.0f) || (cz - a.radius > a.zfar);
    for (int p = 0; p < 4 && !skip; ++p) {
        const float dd = a.plane[p][0] * cx + a.plane[p][1] * cy + a.plane[p][2] * cz;
        if (dd < -a.radius) skip = true;
    }
    if (skip) return;
    const float hi = (float)b[2];
    const int slot = atomicAdd(a.list.count, 1);
    a.list.tile[slot] = t;
    a.list.base[slot] = make_float4((float)b[0], (float)b[1], hi, (float)(b[2] - (double)hi));
}

template <typename T>
__device__ __forceinline__ bool same_bits(T x, T y)
{
    unsigned bx = 0u, by = 0u;
    memcpy(&bx, &x, sizeof(T));
    memcpy(&by, &y, sizeof(T));
    return bx == by;
}

// Fusion of the listed tiles; a fixed grid of CTAs walks the list.  Thread
// (tx, ty) of a tile owns the column of TZ nodes (i0 + tx, j0 + ty, k0 + dz).
// With a cell view, a tile where some node's stored value changed is stamped
// with the fusion counter (by every thread that changed one: the same value);
// a fused node whose value stays -- free space seen again, still outside the
// band -- changes only its weight, which no cell record holds, so its tile's
// records need no rewrite.
template <typename TS, typename TW>
__global__ void __launch_bounds__(TX * TY, 4) integrate_kernel(IntegArgs a)
{
    TS* const tsdf = static_cast<TS*>(a.tsdf);
    TW* const weight = static_cast<TW*>(a.weight);
    const int n_active = *a.list.count;
    const int stamp = a.tile_stamp ? *a.stamp_dev : 0;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float ai[3] = {a.list.step[0], a.list.step[1], a.list.step[2]};
    const float aj[3] = {a.list.step[3], a.list.step[4], a.list.step[5]};
    const float ak[3] = {a.list.step[6], a.list.step[7], a.list.step[8]};
    const float lx = fmaf((float)tx, ai[0], (float)ty * aj[0]);
    const float ly = fmaf((float)tx, ai[1], (float)ty * aj[1]);
    const float lz = fmaf((float)tx, ai[2], (float)ty * aj[2]);
    const size_t plane_stride = (size_t)a.nx * a.ny;
    for (int e = blockIdx.x; e < n_active; e += gridDim.x) {
        const int t = a.list.tile[e];
        const float4 base = a.list.base[e];
        const int bx = t % a.tiles[0], by = (t / a.tiles[0]) % a.tiles[1], bz = t / (a.tiles[0] * a.tiles[1]);
        const int i = bx * TX + tx, j = by * TY + ty, k0 = bz * TZ;
        if (i >= a.nx || j >= a.ny) continue;
        const float bx_ = base.x, by_ = base.y, bz_hi = base.z, bz_lo = base.w;
        size_t idx = (size_t)i + (size_t)a.nx * j + plane_stride * k0;
        bool changed = false;
        for (int dz = 0; dz < TZ; ++dz, idx += plane_stride) {
            const int k = k0 + dz;
            if (k >= a.nz) break;
            const float fz = (float)dz;
            const float xc = bx_ + fmaf(fz, ak[0], lx);
            const float yc = by_ + fmaf(fz, ak[1], ly);
            const float zl = bz_lo + fmaf(fz, ak[2], lz);
            const float zc = bz_hi + zl;
            if (!(zc > 0.0f)) continue;
            const float inv = __frcp_rn(zc);
            const float u = fmaf(a.cam.fx * xc, inv, a.cam.cx);
            const float v = fmaf(a.cam.fy * yc, inv, a.cam.cy);
            const float uf = floorf(u + 0.5f), vf = floorf(v + 0.5f);
            if (!(uf >= 0.0f && uf < (float)a.cam.width && vf >= 0.0f && vf < (float)a.cam.height)) continue;
            const float d = __ldg(a.depth + (size_t)vf * a.cam.width + (size_t)uf);
            if (!pf_depth_usable(d, a.cam.dmin, a.cam.dmax)) continue;
            const float sdf = (d - bz_hi) - zl;
            if (sdf < -a.trunc) continue;
            const float tt = fminf(1.0f, __fdiv_rn(sdf, a.trunc));
            const float w = pf_to_float(weight[idx]);
            const TS old = tsdf[idx];
            float tn = tt;
            if (w > 0.0f) tn = __fdiv_rn(fmaf(w, pf_decode(pf_to_float(old)), tt), w + 1.0f);
            const float wn = fminf(w + 1.0f, a.max_weight);
            const TS stored = pf_from_float<TS>(pf_encode(tn, wn));
            changed = changed || !same_bits(stored, old);
            tsdf[idx] = stored;
            weight[idx] = pf_from_float<TW>(wn);
        }
        if (changed && a.tile_stamp) a.tile_stamp[t] = stamp;
    }
}

template <typename TS, typename TW>
__global__ void fill_kernel(void* tsdf_, void* weight_, size_t n)
{
    TS* tsdf = static_cast<TS*>(tsdf_);
    TW* weight = static_cast<TW*>(weight_);
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t step = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += step) {
        tsdf[i] = pf_from_float<TS>(PF_UNOBSERVED);
        weight[i] = pf_from_float<TW>(0.0f);
    }
}

// Cell view: for every cell (lower corner node i, j, k) its eight encoded
// corner values with the x-differences the interpolation needs already
// formed: float4 (v000, v100 - v000, v010, v110 - v010) and float4 (v001,
// v101 - v001, v011, v111 - v011).  The subtraction is the same float
// operation the fitness would do, so results are bit-identical, and a
// non-finite corner still makes the interpolated value non-finite.  A cell
// depends on the nodes of its own fusion tile and of the next tiles along
// +x, +y, +z, so a tile is rewritten when a node value of any of those was
// changed by the last fusion (or always, after a reset or upload).
struct RefreshArgs {
    const void* tsdf;
    void* cells;
    float* cells32;  // 16-/8-bit grids, full view: the float records as well
    int nx, ny, nz;
    const int* tile_stamp;
    const int* stamp_dev;
    int all;
    int tiles[3];
    FusionList list;  // list.refresh_tile / count[1]: the tiles to rewrite
};

// One thread per tile: a tile's cells are rewritten when the tile or one of
// its neighbours along +x, +y, +z (whose nodes its cells reach) had a node
// value changed by the last fusion, or always (all).  Order of the list as in
// fusion_tiles_kernel: any, with the same result.
__global__ void __launch_bounds__(256) refresh_tiles_kernel(RefreshArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_tiles = a.tiles[0] * a.tiles[1] * a.tiles[2];
    if (t >= n_tiles) return;
    const int bx = t % a.tiles[0], by = (t / a.tiles[0]) % a.tiles[1], bz = t / (a.tiles[0] * a.tiles[1]);
    bool need = a.all != 0;
    const int stamp = *a.stamp_dev;
    for (int q = 0; q < 8 && !need; ++q) {
        const int x = bx + (q & 1), y = by + ((q >> 1) & 1), z = bz + (q >> 2);
        if (x < a.tiles[0] && y < a.tiles[1] && z < a.tiles[2])
            need = a.tile_stamp[x + a.tiles[0] * (y + (size_t)a.tiles[1] * z)] == stamp;
    }
    if (need) a.list.refresh_tile[atomicAdd(a.list.count + 1, 1)] = t;
}

// One cell-view record.  Float storage: two float4 holding the corners with
// the x-differences precomputed (v000, v100 - v000, v010, v110 - v010 |
// v001, v101 - v001, v011, v111 - v011).  16-bit storage: the eight corner
// values as stored (v000, v100, v010, v110 | v001, v101, v011, v111), one
// 16-byte record; the reader forms the differences in float, so the fitness
// sees exactly the stored grid (a difference rounded to 16 bits would not be).
__device__ inline void store_cell(const float* p, size_t nx, size_t nxy, float* cells, size_t idx)
{
    const float v000 = p[0], v010 = p[nx], v001 = p[nxy], v011 = p[nxy + nx];
    float4* c = reinterpret_cast<float4*>(cells) + 2 * idx;
    c[0] = make_float4(v000, p[1] - v000, v010, p[nx + 1] - v010);
    c[1] = make_float4(v001, p[nxy + 1] - v001, v011, p[nxy + nx + 1] - v011);
}

template <typename T>
__device__ inline void store_cell(const T* p, size_t nx, size_t nxy, T* cells, size_t idx)
{
    static_assert(sizeof(T) == 2 || sizeof(T) == 1, "16- or 8-bit storage");
    const T h[8] = {p[0], p[1], p[nx], p[nx + 1], p[nxy], p[nxy + 1], p[nxy + nx], p[nxy + nx + 1]};
    if (sizeof(T) == 2)
        reinterpret_cast<uint4*>(cells)[idx] = *reinterpret_cast<const uint4*>(h);
    else
        reinterpret_cast<uint2*>(cells)[idx] = *reinterpret_cast<const uint2*>(h);
}

// The float record of a 16-bit grid: the stored values converted exactly and
// the x-differences formed in float, as the 16-bit reader forms them, so both
// records of a cell give bit-identical samples.
template <typename T>
__device__ inline void store_cell32(const T* p, size_t nx, size_t nxy, float* cells32, size_t idx)
{
    const float v000 = pf_to_float(p[0]), v010 = pf_to_float(p[nx]), v001 = pf_to_float(p[nxy]),
                v011 = pf_to_float(p[nxy + nx]);
    float4* c = reinterpret_cast<float4*>(cells32) + 2 * idx;
    c[0] = make_float4(v000, pf_to_float(p[1]) - v000, v010, pf_to_float(p[nx + 1]) - v010);
    c[1] = make_float4(v001, pf_to_float(p[nxy + 1]) - v001, v011, pf_to_float(p[nxy + nx + 1]) - v011);
}

// A float grid's node values rounded once into a narrower view (the search
// view of a float master grid): the eight corners converted with the
// storage rule (a value that rounds to +-1 becomes the outside-the-band
// code), written as the narrow record, and with a full view also as the
// float record formed from the rounded values -- the grid the search reads.
template <typename TV>
__device__ inline void store_cell_rounded(const float* p, size_t nx, size_t nxy, TV* cells, float* cells32,
                                          size_t idx)
{
    static_assert(sizeof(TV) == 2 || sizeof(TV) == 1, "16- or 8-bit view");
    const TV h[8] = {pf_from_float<TV>(p[0]),       pf_from_float<TV>(p[1]),        pf_from_float<TV>(p[nx]),
                     pf_from_float<TV>(p[nx + 1]),  pf_from_float<TV>(p[nxy]),      pf_from_float<TV>(p[nxy + 1]),
                     pf_from_float<TV>(p[nxy + nx]), pf_from_float<TV>(p[nxy + nx + 1])};
    if (sizeof(TV) == 2)
        reinterpret_cast<uint4*>(cells)[idx] = *reinterpret_cast<const uint4*>(h);
    else
        reinterpret_cast<uint2*>(cells)[idx] = *reinterpret_cast<const uint2*>(h);
    if (cells32) {
        float v[8];
        for (int c = 0; c < 8; ++c) v[c] = pf_to_float(h[c]);
        float4* c = reinterpret_cast<float4*>(cells32) + 2 * idx;
        c[0] = make_float4(v[0], v[1] - v[0], v[2], v[3] - v[2]);
        c[1] = make_float4(v[4], v[5] - v[4], v[6], v[7] - v[6]);
    }
}

// TS: storage of the node array; TV: storage of the view (TS itself, or a
// narrower type for the search view of a float grid).  A fixed grid of CTAs
// walks the list of tiles to rewrite.
template <typename TS, typename TV>
__global__ void __launch_bounds__(TX * TY, 4) cells_refresh_kernel(RefreshArgs a)
{
    const int n_list = a.list.count[1];
    const TS* tsdf = static_cast<const TS*>(a.tsdf);
    TV* cells = static_cast<TV*>(a.cells);
    const size_t nx = a.nx, nxy = (size_t)a.nx * a.ny;
    for (int e = blockIdx.x; e < n_list; e += gridDim.x) {
        const int t = a.list.refresh_tile[e];
        const int bx = t % a.tiles[0], by = (t / a.tiles[0]) % a.tiles[1], bz = t / (a.tiles[0] * a.tiles[1]);
        const int i = bx * TX + threadIdx.x, j = by * TY + threadIdx.y;
        if (i >= a.nx - 1 || j >= a.ny - 1) continue;
        for (int dz = 0; dz < TZ; ++dz) {
            const int k = bz * TZ + dz;
            if (k >= a.nz - 1) break;
            const size_t idx = i + nx * j + nxy * k;
            if constexpr (!std::is_same<TS, TV>::value) {
                store_cell_rounded(tsdf + idx, nx, nxy, cells, a.cells32, idx);
            } else {
                store_cell(tsdf + idx, nx, nxy, cells, idx);
                if constexpr (!std::is_same<TS, float>::value)
                    if (a.cells32) store_cell32(tsdf + idx, nx, nxy, a.cells32, idx);
            }
        }
    }
}

// CTAs of the list-walking fusion and refresh kernels: 4 per SM.
int list_ctas(int device)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 152;
    return 4 * sms;
}

pf_status enqueue_refresh(pf_volume* v, cudaStream_t s, int all)
{
    if (!v->cells) return PF_OK;
    RefreshArgs r;
    r.tsdf = v->tsdf;
    r.cells = v->cells;
    r.cells32 = v->cells32;
    r.nx = v->desc.nx;
    r.ny = v->desc.ny;
    r.nz = v->desc.nz;
    const int n_tiles = v->tiles[0] * v->tiles[1] * v->tiles[2];
    r.tile_stamp = v->tile_stamp;
    r.stamp_dev = v->tile_stamp + n_tiles;
    r.all = all;
    for (int q = 0; q < 3; ++q) r.tiles[q] = v->tiles[q];
    r.list = v->list;
    if (all) {  // outside a fusion: the list counter was not reset by fusion_begin_kernel
        fusion_begin_kernel<<<1, 32, 0, s>>>(v->list, nullptr);
        pf::count_launch();
    }
    refresh_tiles_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(r);
    pf::count_launch();
    const int grid = list_ctas(v->device);
    const dim3 blk(TX, TY);
    if (v->desc.tsdf_dtype != pf_view_dtype(v)) {  // the search view of a float grid
        switch (pf_view_dtype(v)) {
        case PF_F16: cells_refresh_kernel<float, __half><<<grid, blk, 0, s>>>(r); break;
        case PF_BF16: cells_refresh_kernel<float, __nv_bfloat16><<<grid, blk, 0, s>>>(r); break;
        default: cells_refresh_kernel<float, __nv_fp8_e4m3><<<grid, blk, 0, s>>>(r); break;
        }
    } else {
        switch (v->desc.tsdf_dtype) {
        case PF_F16: cells_refresh_kernel<__half, __half><<<grid, blk, 0, s>>>(r); break;
        case PF_BF16: cells_refresh_kernel<__nv_bfloat16, __nv_bfloat16><<<grid, blk, 0, s>>>(r); break;
        case PF_FP8E4M3: cells_refresh_kernel<__nv_fp8_e4m3, __nv_fp8_e4m3><<<grid, blk, 0, s>>>(r); break;
        default: cells_refresh_kernel<float, float><<<grid, blk, 0, s>>>(r); break;
        }
    }
    pf::count_launch();
    PF_LAUNCHED();
    return PF_OK;
}

// Launch a kernel templated on (tsdf storage, weight storage) for volume v.
template <template <typename, typename> class K, typename... Args>
void dispatch_storage(const pf_volume* v, Args&&... args)
{
    const bool u8 = v->desc.weight_u8 != 0;
    switch (v->desc.tsdf_dtype) {
    case PF_F16:
        if (u8) K<__half, uint8_t>::run(args...); else K<__half, float>::run(args...);
        break;
    case PF_BF16:
        if (u8) K<__nv_bfloat16, uint8_t>::run(args...); else K<__nv_bfloat16, float>::run(args...);
        break;
    case PF_FP8E4M3:
        if (u8) K<__nv_fp8_e4m3, uint8_t>::run(args...); else K<__nv_fp8_e4m3, float>::run(args...);
        break;
    default:
        if (u8) K<float, uint8_t>::run(args...); else K<float, float>::run(args...);
        break;
    }
}

template <typename TS, typename TW>
struct FillLaunch {
    static void run(void* tsdf, void* weight, size_t n, cudaStream_t s)
    {
        fill_kernel<TS, TW><<<152 * 8, 256, 0, s>>>(tsdf, weight, n);
    }
};

template <typename TS, typename TW>
struct IntegrateLaunch {
    static void run(int grid, const IntegArgs& a, cudaStream_t s)
    {
        integrate_kernel<TS, TW><<<grid, dim3(TX, TY), 0, s>>>(a);
    }
};

pf_status check_desc(const pf_volume_desc* d)
{
    if (!d) return PF_ERR_INVALID_ARG;
    if (d->nx < 2 || d->ny < 2 || d->nz < 2 || d->nx > 4096 || d->ny > 4096 || d->nz > 4096)
        return PF_ERR_INVALID_ARG;
    if ((double)d->nx * d->ny * d->nz >= 2147483648.0) return PF_ERR_INVALID_ARG;
    if (!(d->voxel_size > 0.0f) || !(d->trunc > 0.0f) || !std::isfinite(d->voxel_size) || !std::isfinite(d->trunc))
        return PF_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d->origin[a])) return PF_ERR_INVALID_ARG;
    if (d->max_weight < 1 || d->max_weight > 65535) return PF_ERR_INVALID_ARG;
    if (d->cell_view < -1 || d->cell_view > 2) return PF_ERR_INVALID_ARG;
    if (d->weight_u8 != 0 && d->weight_u8 != 1) return PF_ERR_INVALID_ARG;
    if (d->weight_u8 && d->max_weight > 255) return PF_ERR_INVALID_ARG;
    if (d->tsdf_dtype != PF_F32 && d->tsdf_dtype != PF_F16 && d->tsdf_dtype != PF_BF16 &&
        d->tsdf_dtype != PF_FP8E4M3)
        return PF_ERR_UNSUPPORTED;
    // a search view narrower than the storage: float grids only, and it
    // needs a cell view
    if (d->search_dtype != PF_F32 && d->search_dtype != d->tsdf_dtype) {
        if (d->search_dtype != PF_F16 && d->search_dtype != PF_BF16 && d->search_dtype != PF_FP8E4M3)
            return PF_ERR_UNSUPPORTED;
        if (d->tsdf_dtype != PF_F32) return PF_ERR_UNSUPPORTED;
        if (d->cell_view == -1) return PF_ERR_INVALID_ARG;
    }
    return PF_OK;
}

pf_status enqueue_reset(pf_volume* v, cudaStream_t s)
{
    dispatch_storage<FillLaunch>(v, v->tsdf, v->weight, v->n_nodes, s);
    pf::count_launch();
    PF_LAUNCHED();
    return enqueue_refresh(v, s, 1);
}

void free_list(FusionList& l)
{
    cudaFree(l.count);
    cudaFree(l.tile);
    cudaFree(l.base);
    cudaFree(l.step);
    cudaFree(l.refresh_tile);
    l = FusionList();
}

bool finite_pose(const double* P)
{
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(P[i])) return false;
    return true;
}

}  // namespace

extern "C" {

pf_status pf_create_volume(const pf_volume_desc* desc, void* stream, pf_volume** out)
{
    if (!out) return PF_ERR_INVALID_ARG;
    *out = nullptr;
    pf_status st = check_desc(desc);
    if (st != PF_OK) return st;
    pf_volume* v = new pf_volume();
    v->desc = *desc;
    v->n_nodes = (size_t)desc->nx * desc->ny * desc->nz;
    v->tiles[0] = (desc->nx + TX - 1) / TX;
    v->tiles[1] = (desc->ny + TY - 1) / TY;
    v->tiles[2] = (desc->nz + TZ - 1) / TZ;
    const size_t ts = pf_dtype_size(desc->tsdf_dtype), ws = desc->weight_u8 ? 1 : 4;
    const pf_dtype vdt = pf_view_dtype(v);
    const size_t vs = pf_dtype_size(vdt);
    // the full view of a 16-/8-bit grid keeps both its narrow records (lanes
    // on points: two or four records per sector) and float records (lanes on
    // particles: no conversions); the narrow view keeps the narrow records
    // only; a float grid has the float records only
    const size_t bytes32 = vdt == PF_F32 ? 0 : v->n_nodes * 32;
    const size_t view_bytes = v->n_nodes * 8 * vs;
    const size_t grid_bytes = v->n_nodes * (ts + ws);
    cudaError_t e = cudaGetDevice(&v->device);
    int mode = desc->cell_view;
    if (mode == 0) {
        // auto, within half of the device memory free now: the full view
        // when it fits (decoding narrow records on load slows the search
        // once the particles converge), else the narrow one, else none
        size_t free_b = 0, total_b = 0;
        if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
        const size_t budget = free_b / 2;
        mode = grid_bytes + view_bytes + bytes32 <= budget ? 1 : grid_bytes + view_bytes <= budget ? 2 : -1;
    }
    if (mode == 2 && !bytes32) mode = 1;
    if (mode == -1 && vdt != desc->tsdf_dtype) e = cudaErrorMemoryAllocation;  // no room for the search view
    const bool view = mode >= 1;
    const bool wide = mode == 1;
    if (e == cudaSuccess) e = pf::dev_malloc(&v->tsdf, v->n_nodes * ts);
    if (e == cudaSuccess) e = pf::dev_malloc(&v->weight, v->n_nodes * ws);
    if (e == cudaSuccess && view) e = pf::dev_malloc(&v->cells, view_bytes);
    if (e == cudaSuccess && wide && bytes32) e = pf::dev_malloc(&v->cells32, bytes32);
    const size_t n_tiles = (size_t)v->tiles[0] * v->tiles[1] * v->tiles[2];
    if (e == cudaSuccess) e = pf::dev_malloc(&v->list.count, 2 * sizeof(int));
    if (e == cudaSuccess) e = pf::dev_malloc(&v->list.tile, n_tiles * sizeof(int));
    if (e == cudaSuccess) e = pf::dev_malloc(&v->list.base, n_tiles * sizeof(float4));
    if (e == cudaSuccess) e = pf::dev_malloc(&v->list.step, 9 * sizeof(float));
    if (e == cudaSuccess && view) e = pf::dev_malloc(&v->list.refresh_tile, n_tiles * sizeof(int));
    if (e == cudaSuccess && view)
        e = pf::dev_malloc(&v->tile_stamp, sizeof(int) * ((size_t)v->tiles[0] * v->tiles[1] * v->tiles[2] + 1));
    if (e == cudaSuccess && view)
        e = cudaMemset(v->tile_stamp, 0, sizeof(int) * ((size_t)v->tiles[0] * v->tiles[1] * v->tiles[2] + 1));
    if (e != cudaSuccess) {
        cudaFree(v->tsdf);
        cudaFree(v->weight);
        cudaFree(v->cells);
        cudaFree(v->cells32);
        cudaFree(v->tile_stamp);
        free_list(v->list);
        delete v;
        cudaGetLastError();
        return pf::cuda_status(e);
    }
    st = enqueue_reset(v, (cudaStream_t)stream);
    if (st != PF_OK) {
        pf_destroy_volume(v);
        return st;
    }
    *out = v;
    return PF_OK;
}

pf_status pf_destroy_volume(pf_volume* v)
{
    if (!v) return PF_OK;
    cudaDeviceSynchronize();
    pf::align_release(v);
    cudaFree(v->tsdf);
    cudaFree(v->weight);
    cudaFree(v->cells);
    cudaFree(v->cells32);
    cudaFree(v->tile_stamp);
    free_list(v->list);
    pf_workspace& w = v->ws;
    cudaFree(w.points);
    cudaFree(w.block_counts);
    cudaFree(w.n_points);
    cudaFree(w.part_S);
    cudaFree(w.part_C);
    cudaFree(w.chunks);
    cudaFree(w.point_tile);
    cudaFree(w.kept);
    cudaFree(w.kept_count);
    cudaFree(w.order_scratch);
    cudaFree(w.chunk_counter);
    cudaFree(w.chunk_E);
    cudaFree(w.chunk_C);
    cudaFree(w.counter);
    cudaFree(w.state);
    cudaFree(w.pose_in);
    cudaFree(w.pose_out);
    cudaFree(w.stats);
    delete v;
    return PF_OK;
}

static pf_status pf_reset_volume_impl(pf_volume* v, void* stream)
{
    if (!v) return PF_ERR_INVALID_ARG;
    return enqueue_reset(v, (cudaStream_t)stream);
}

static pf_status pf_set_fitness_variant_impl(pf_volume* v, int variant)
{
    if (!v || variant < 0 || variant > 11 || (variant & 3) == 3 && !v->cells) return PF_ERR_INVALID_ARG;
    // the plain baseline exists for float tsdf and float weights only
    if ((variant & 3) == 1 && (v->desc.tsdf_dtype != PF_F32 || v->desc.weight_u8)) return PF_ERR_INVALID_ARG;
    v->fitness_variant = variant;
    return PF_OK;
}

pf_status pf_volume_info(const pf_volume* v, unsigned long long* storage_bytes, int* cell_view)
{
    if (!v) return PF_ERR_INVALID_ARG;
    const size_t n = v->n_nodes, ts = pf_dtype_size(v->desc.tsdf_dtype), vs = pf_dtype_size(pf_view_dtype(v));
    const size_t n_tiles = (size_t)v->tiles[0] * v->tiles[1] * v->tiles[2];
    size_t b = n * ts + n * (v->desc.weight_u8 ? 1 : 4);
    if (v->cells) b += n * 8 * vs + sizeof(int) * (n_tiles + 1);
    if (v->cells32) b += n * 32;
    if (storage_bytes) *storage_bytes = b;
    if (cell_view) *cell_view = !v->cells ? -1 : (v->cells32 || pf_view_dtype(v) == PF_F32) ? 1 : 2;
    return PF_OK;
}

}  // extern "C"

namespace {

// Host-side conversion of one encoded value to and from the storage type.
void store_host(pf_dtype dt, float e, unsigned char* dst)
{
    switch (dt) {
    case PF_F16: { const __half h = pf_from_float<__half>(e); std::memcpy(dst, &h, 2); break; }
    case PF_BF16: { const __nv_bfloat16 h = pf_from_float<__nv_bfloat16>(e); std::memcpy(dst, &h, 2); break; }
    case PF_FP8E4M3: { const __nv_fp8_e4m3 h = pf_from_float<__nv_fp8_e4m3>(e); std::memcpy(dst, &h, 1); break; }
    default: std::memcpy(dst, &e, 4); break;
    }
}

float load_host(pf_dtype dt, const unsigned char* src)
{
    switch (dt) {
    case PF_F16: { __half h; std::memcpy(&h, src, 2); return pf_to_float(h); }
    case PF_BF16: { __nv_bfloat16 h; std::memcpy(&h, src, 2); return pf_to_float(h); }
    case PF_FP8E4M3: { __nv_fp8_e4m3 h; std::memcpy(&h, src, 1); return pf_to_float(h); }
    default: { float f; std::memcpy(&f, src, 4); return f; }
    }
}

}  // namespace

extern "C" {

static pf_status pf_volume_upload_impl(pf_volume* v, const float* tsdf_host, const float* weight_host)
{
    if (!v || !tsdf_host || !weight_host) return PF_ERR_INVALID_ARG;
    const size_t n = v->n_nodes;
    const pf_dtype dt = v->desc.tsdf_dtype;
    const size_t ts = pf_dtype_size(dt);
    std::vector<unsigned char> enc(n * ts);
    std::vector<uint8_t> w8(v->desc.weight_u8 ? n : 0);
    for (size_t i = 0; i < n; ++i) {
        const float w = weight_host[i];
        if (!(w >= 0.0f) || !std::isfinite(w) || w > (float)v->desc.max_weight) return PF_ERR_INVALID_ARG;
        if (w > 0.0f && !(std::fabs(tsdf_host[i]) <= 1.0f)) return PF_ERR_INVALID_ARG;
        if (v->desc.weight_u8 && w != std::floor(w)) return PF_ERR_INVALID_ARG;
        store_host(dt, pf_encode(tsdf_host[i], w), enc.data() + i * ts);
        if (v->desc.weight_u8) w8[i] = (uint8_t)w;
    }
    PF_CUDA(cudaDeviceSynchronize());
    PF_CUDA(cudaMemcpy(v->tsdf, enc.data(), n * ts, cudaMemcpyHostToDevice));
    if (v->desc.weight_u8) PF_CUDA(cudaMemcpy(v->weight, w8.data(), n, cudaMemcpyHostToDevice));
    else PF_CUDA(cudaMemcpy(v->weight, weight_host, n * 4, cudaMemcpyHostToDevice));
    pf_status st = enqueue_refresh(v, 0, 1);
    if (st != PF_OK) return st;
    PF_CUDA(cudaDeviceSynchronize());
    return PF_OK;
}

static pf_status pf_volume_download_impl(const pf_volume* v, float* tsdf_host, float* weight_host)
{
    if (!v || !tsdf_host || !weight_host) return PF_ERR_INVALID_ARG;
    const size_t n = v->n_nodes;
    const pf_dtype dt = v->desc.tsdf_dtype;
    const size_t ts = pf_dtype_size(dt);
    PF_CUDA(cudaDeviceSynchronize());
    if (dt == PF_F32) {
        PF_CUDA(cudaMemcpy(tsdf_host, v->tsdf, n * 4, cudaMemcpyDeviceToHost));
    } else {
        std::vector<unsigned char> raw(n * ts);
        PF_CUDA(cudaMemcpy(raw.data(), v->tsdf, n * ts, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) tsdf_host[i] = load_host(dt, raw.data() + i * ts);
    }
    if (v->desc.weight_u8) {
        std::vector<uint8_t> w8(n);
        PF_CUDA(cudaMemcpy(w8.data(), v->weight, n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) weight_host[i] = (float)w8[i];
    } else {
        PF_CUDA(cudaMemcpy(weight_host, v->weight, n * 4, cudaMemcpyDeviceToHost));
    }
    for (size_t i = 0; i < n; ++i)
        tsdf_host[i] = weight_host[i] > 0.0f ? pf_decode(tsdf_host[i]) : 1.0f;
    return PF_OK;
}

}  // extern "C"

namespace {

pf_status integrate_impl(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr, const double* P_host,
                         const double* P_dev, cudaStream_t s)
{
    if (!v || !depth_dev) return PF_ERR_INVALID_ARG;
    pf_status st = pf::check_intrinsics(intr);
    if (st != PF_OK) return st;
    const pf_volume_desc& d = v->desc;
    IntegArgs a;
    a.tsdf = v->tsdf;
    a.weight = v->weight;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.trunc = d.trunc;
    a.max_weight = (float)d.max_weight;
    a.cam = make_cam(intr);
    a.depth = depth_dev;
    a.pose_dev = P_dev;
    for (int q = 0; q < 12; ++q) a.pose[q] = P_host ? P_host[q] : 0.0;
    for (int q = 0; q < 3; ++q) a.origin[q] = d.origin[q];
    a.vs = d.voxel_size;
    // side planes through the camera centre: pixel range u in [-0.5, W - 0.5)
    const double lx0 = (-0.5 - intr->cx) / intr->fx, lx1 = (intr->width - 0.5 - intr->cx) / intr->fx;
    const double ly0 = (-0.5 - intr->cy) / intr->fy, ly1 = (intr->height - 0.5 - intr->cy) / intr->fy;
    const double pl[4][3] = {{1.0, 0.0, -lx0}, {-1.0, 0.0, lx1}, {0.0, 1.0, -ly0}, {0.0, -1.0, ly1}};
    for (int p = 0; p < 4; ++p) {
        double n = sqrt(pl[p][0] * pl[p][0] + pl[p][1] * pl[p][1] + pl[p][2] * pl[p][2]);
        for (int c = 0; c < 3; ++c) a.plane[p][c] = (float)(pl[p][c] / n);
    }
    a.zfar = d.trunc + intr->depth_max;
    const double vs = d.voxel_size;
    a.radius = (float)(0.5 * vs * sqrt((double)((TX - 1) * (TX - 1) + (TY - 1) * (TY - 1) + (TZ - 1) * (TZ - 1)))
                       + 0.01 * vs + 1e-3);
    // the fusion counter lives on the device (after the per-tile stamps), so
    // a captured and replayed launch sequence still marks each fusion apart
    const int n_tiles = v->tiles[0] * v->tiles[1] * v->tiles[2];
    a.tile_stamp = v->tile_stamp;
    a.stamp_dev = v->tile_stamp ? v->tile_stamp + n_tiles : nullptr;
    for (int q = 0; q < 3; ++q) a.tiles[q] = v->tiles[q];
    a.list = v->list;
    ++v->stamp;
    pf::timing_begin(pf::KC_INTEGRATE, s);
    fusion_begin_kernel<<<1, 32, 0, s>>>(v->list, v->tile_stamp ? v->tile_stamp + n_tiles : nullptr);
    fusion_tiles_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(a);
    dispatch_storage<IntegrateLaunch>(v, list_ctas(v->device), a, s);
    pf::count_launch(3);
    pf::timing_end(pf::KC_INTEGRATE, s);
    PF_LAUNCHED();
    pf::timing_begin(pf::KC_REFRESH, s);
    st = enqueue_refresh(v, s, 0);
    pf::timing_end(pf::KC_REFRESH, s);
    return st;
}

__global__ void compose_kernel(const double* A, const double* B, double* out)
{
    const int t = threadIdx.x;
    if (t < 16) {
        const int r = t >> 2, c = t & 3;
        double acc = 0.0;
        for (int m = 0; m < 4; ++m) acc += A[4 * r + m] * B[4 * m + c];
        out[t] = acc;
    }
}

}  // namespace

extern "C" {

static pf_status pf_integrate_impl(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr,
                                   const double P[16], void* stream)
{
    if (!P || !finite_pose(P)) return PF_ERR_INVALID_ARG;
    return integrate_impl(v, depth_dev, intr, P, nullptr, (cudaStream_t)stream);
}

static pf_status pf_integrate_async_impl(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr,
                                         const double* P_dev, void* stream)
{
    if (!P_dev) return PF_ERR_INVALID_ARG;
    return integrate_impl(v, depth_dev, intr, nullptr, P_dev, (cudaStream_t)stream);
}

pf_status pf_pose_compose(const double* a_dev, const double* b_dev, double* out_dev, void* stream)
{
    if (!a_dev || !b_dev || !out_dev || out_dev == a_dev || out_dev == b_dev) return PF_ERR_INVALID_ARG;
    compose_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(a_dev, b_dev, out_dev);
    pf::count_launch();
    PF_LAUNCHED();
    return PF_OK;
}

}  // extern "C"

// Every entry point that takes a volume keeps its last failing status
// there (pf_volume_last_error).
extern "C" {

pf_status pf_volume_last_error(pf_volume* v, int clear)
{
    if (!v) return PF_ERR_INVALID_ARG;
    const pf_status s = v->last_status;
    if (clear) v->last_status = PF_OK;
    return s;
}

pf_status pf_reset_volume(pf_volume* v, void* stream)
{
    return pf::keep_status(v, pf_reset_volume_impl(v, stream));
}

pf_status pf_set_fitness_variant(pf_volume* v, int variant)
{
    return pf::keep_status(v, pf_set_fitness_variant_impl(v, variant));
}

pf_status pf_volume_upload(pf_volume* v, const float* tsdf_host, const float* weight_host)
{
    return pf::keep_status(v, pf_volume_upload_impl(v, tsdf_host, weight_host));
}

pf_status pf_volume_download(const pf_volume* v, float* tsdf_host, float* weight_host)
{
    return pf::keep_status(v, pf_volume_download_impl(v, tsdf_host, weight_host));
}

pf_status pf_integrate(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr, const double P[16],
                       void* stream)
{
    return pf::keep_status(v, pf_integrate_impl(v, depth_dev, intr, P, stream));
}

pf_status pf_integrate_async(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr, const double* P_dev,
                             void* stream)
{
    return pf::keep_status(v, pf_integrate_async_impl(v, depth_dev, intr, P_dev, stream));
}

}  // extern "C"
