// Back-projection, fitness gather-reduce and the randomized pose search.
//
// Randomized optimization (Sec. III-B): in iteration i, K delta poses are
// drawn within the search size s = (omega deg, v cm) -- here the pre-drawn
// templates u_k scaled by s -- and applied to the current pose, dP_k * P.
// Each candidate is scored by the fitness
//     E_k = (1/|X_k|) sum_{x in X_k} |tsdf(dP_k P x)|
// (tsdf stored divided by tau), the advantage set {k : E_k < E(P)} is
// averaged (rotation vectors and translations) into the update of P, and
// s <- beta s + (1 - beta) E(P_new) s.
//
// GPU design
//   * fitness_kernel is the hot loop.  Grid = (particle chunks) x (point
//     tiles).  A CTA builds its chunk's KC transforms in shared memory
//     (already scaled to grid units), keeps PPT points per thread in
//     registers, and for each particle lets the 32 lanes of a warp evaluate
//     32 consecutive image points: neighbouring pixels land in neighbouring
//     voxels, so the eight corner gathers of a warp fall in a handful of
//     cache lines.  Per-particle sums are reduced with warp shuffles into
//     per-warp shared accumulators, then per CTA into (S, C) partials in a
//     fixed order -- no floating-point atomics, bit-reproducible.  When the
//     chunk's particles nearly coincide, lanes take particles instead and
//     share each point through shared memory.
//   * Samples go in pairs through Blackwell's packed f32x2 FMA / add (two
//     float operations per instruction, rounded exactly as two scalar ones).
//     A point whose samples under every particle of the chunk provably stay
//     inside the grid skips the per-axis range test and forms its cell index
//     as one linear combination.  A float cell-view record (32 bytes) is one
//     256-bit load.
//   * The last CTA to finish (ticket counter, no spinning) reduces the
//     partials over point tiles and, for the search, does the selection:
//     argmin (lowest index on ties), advantage set, its mean, the FP64 pose
//     composition with re-orthonormalisation and the search-size update.
//     One launch per iteration therefore carries the whole iteration; the
//     paper's mean update adds one single-particle launch for E(P_new).
//   * Everything stays on the device: a frame is a fixed sequence of
//     launches with no host round trip, so it can be captured in a graph.
#include <float.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>
#include <vector>

#include "pf_internal.cuh"
#include "ptiles.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Search state kept in device memory between the launches of one frame.
// ---------------------------------------------------------------------------
struct SearchState {
    double P[12];     // current pose, row-major 3x4 camera-to-world
    double P0[12];    // initial pose
    double s[2];      // search size (deg, cm) of the current iteration
    int lost;         // frame declared lost
    int pending_s;    // mean update: s waits for E(P_new)
    int n_points;
    int pad;
};

// ---------------------------------------------------------------------------
// Back-projection (Sec. III, problem setting)
//
// Points are compacted in tile order: the image is cut into 8 x 4-pixel tiles,
// taken row-major over tiles and row-major inside a tile, so 32 consecutive
// points form one compact image patch -- exactly what a warp of the fitness
// kernel evaluates together when points share the lanes, which keeps the
// cells those 32 samples touch close together.  Down-sampling keeps every
// n-th point of this order.  One warp per tile: a ballot gives the tile's
// valid pixels and their ranks.
// ---------------------------------------------------------------------------
constexpr int TILE_W = 8, TILE_H = 4;
constexpr int BP_THREADS = 256, BP_TILES_PER_WARP = 8;
constexpr int BP_CHUNK_TILES = (BP_THREADS / 32) * BP_TILES_PER_WARP;  // tiles per block

__device__ inline int block_sum_int(int v, int* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    __syncthreads();
    return tot;
}

// Pixel of `lane` in `tile`; true when it lies in the image with a usable depth.
__device__ inline bool bp_pixel(const float* __restrict__ depth, const CamK& cam, int tiles_x, int tile, int lane,
                                int& u, int& v, float& z)
{
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    u = tx * TILE_W + (lane & (TILE_W - 1));
    v = ty * TILE_H + lane / TILE_W;
    z = 0.0f;
    if (u >= cam.width || v >= cam.height) return false;
    z = depth[(size_t)v * cam.width + u];
    return pf_depth_usable(z, cam.dmin, cam.dmax);
}

// Valid pixels of this warp's tiles (a warp-uniform count).
__device__ inline int bp_warp_count(const float* __restrict__ depth, const CamK& cam, int n_tiles, int tiles_x)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int c = 0;
    for (int i = 0; i < BP_TILES_PER_WARP; ++i) {
        const int tile = blockIdx.x * BP_CHUNK_TILES + warp * BP_TILES_PER_WARP + i;
        int u, v;
        float z;
        const bool ok = tile < n_tiles && bp_pixel(depth, cam, tiles_x, tile, lane, u, v, z);
        c += __popc(__ballot_sync(0xffffffffu, ok));
    }
    return c;
}

__global__ void __launch_bounds__(BP_THREADS) bp_count_kernel(const float* __restrict__ depth, CamK cam, int n_tiles,
                                                              int tiles_x, int* block_counts)
{
    __shared__ int sh[32];
    const int c = bp_warp_count(depth, cam, n_tiles, tiles_x);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < BP_THREADS / 32; ++w) tot += sh[w];
        block_counts[blockIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(BP_THREADS) bp_write_kernel(const float* __restrict__ depth, CamK cam, int n_tiles,
                                                              int tiles_x, const int* __restrict__ block_counts,
                                                              float4* __restrict__ pts, int* n_out, int* tile_out)
{
    __shared__ int sh[32];
    __shared__ int warp_off[BP_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // points of the earlier blocks
    int off = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) off += block_counts[b];
    off = block_sum_int(off, sh);
    // exclusive scan of the warps' counts, in warp order (= tile order)
    const int c = bp_warp_count(depth, cam, n_tiles, tiles_x);
    if (lane == 0) warp_off[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < BP_THREADS / 32; ++w) {
            const int t = warp_off[w];
            warp_off[w] = acc;
            acc += t;
        }
    }
    __syncthreads();
    int pos = off + warp_off[warp];
    const unsigned below = (1u << lane) - 1u;
    for (int i = 0; i < BP_TILES_PER_WARP; ++i) {
        const int tile = blockIdx.x * BP_CHUNK_TILES + warp * BP_TILES_PER_WARP + i;
        int u, v;
        float z;
        const bool ok = tile < n_tiles && bp_pixel(depth, cam, tiles_x, tile, lane, u, v, z);
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const float x = __fdiv_rn(((float)u - cam.cx) * z, cam.fx);
            const float y = __fdiv_rn(((float)v - cam.cy) * z, cam.fy);
            pts[pos + __popc(m & below)] = make_float4(x, y, z, 0.0f);
            if (tile_out) tile_out[pos + __popc(m & below)] = tile;
        }
        pos += __popc(m);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *n_out = pos;
}

pf_status enqueue_backproject(const float* depth, const pf_intrinsics* intr, float4* pts, int* block_counts,
                              int* n_out, cudaStream_t s, int* tile_out = nullptr)
{
    const int tiles_x = (intr->width + TILE_W - 1) / TILE_W, tiles_y = (intr->height + TILE_H - 1) / TILE_H;
    const int n_tiles = tiles_x * tiles_y;
    const int blocks = (n_tiles + BP_CHUNK_TILES - 1) / BP_CHUNK_TILES;
    CamK cam = make_cam(intr);
    pf::timing_begin(pf::KC_BACKPROJECT, s);
    bp_count_kernel<<<blocks, BP_THREADS, 0, s>>>(depth, cam, n_tiles, tiles_x, block_counts);
    bp_write_kernel<<<blocks, BP_THREADS, 0, s>>>(depth, cam, n_tiles, tiles_x, block_counts, pts, n_out, tile_out);
    pf::count_launch(2);
    pf::timing_end(pf::KC_BACKPROJECT, s);
    PF_LAUNCHED();
    return PF_OK;
}

// ---------------------------------------------------------------------------
// Decimated point sets in a locality order.
//
// Down-sampling by n keeps the compacted points j = 0, n, 2n, ... (tile
// order).  Taken in that order, the 32 points a warp evaluates together lie
// up to 32 image tiles apart, so under one particle they share no cells and
// each warp-wide record load touches ~32 sectors.  The kept points are
// therefore evaluated in another order: grouped by blocks of SC x SR image
// tiles (about n tiles, ~32 kept points), blocks row-major, and within a block
// by tile row, keeping the order of the kept sequence inside each row.  The
// order is a function of the input alone (counts, minima and a scan: no
// order-dependent atomics), and the set of points is the kept set, so only
// the float summation order of the fitness changes.
// ---------------------------------------------------------------------------
// Strides above this keep the strided reading (their blocks would be large
// and their points sparse anyway).
constexpr int kMaxOrderedStride = 64;

// Scratch slots the ordering needs for an image of `pixels` pixels and any
// stride up to kMaxOrderedStride (blocks x rows <= tiles + tiles_x x rows).
inline size_t kept_slots_bound(size_t pixels) { return pixels / 32 + 2 * 2048 + 4096 + 2048 * 8 + 64; }

struct KeptOrder {
    int stride;          // n > 1
    int tiles_x, sc, sr; // image tiles per row; block of sc x sr tiles
    int blocks_x;        // blocks per row of blocks
    int n_slots;         // blocks x sr
};

inline KeptOrder kept_order(int stride, int width, int height)
{
    KeptOrder o;
    o.stride = stride;
    o.tiles_x = (width + TILE_W - 1) / TILE_W;
    const int tiles_y = (height + TILE_H - 1) / TILE_H;
    o.sc = std::max(1, (int)std::ceil(std::sqrt((double)stride)));
    o.sr = std::max(1, (stride + o.sc - 1) / o.sc);
    o.blocks_x = (o.tiles_x + o.sc - 1) / o.sc;
    const int blocks_y = (tiles_y + o.sr - 1) / o.sr;
    o.n_slots = o.blocks_x * blocks_y * o.sr;
    return o;
}

__device__ __forceinline__ void kept_slot(const KeptOrder& o, int tile, int& block, int& row)
{
    const int tx = tile % o.tiles_x, ty = tile / o.tiles_x;
    block = (ty / o.sr) * o.blocks_x + tx / o.sc;
    row = ty % o.sr;
}

__global__ void kept_clear_kernel(int* cnt, int* first, int n_slots)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += gridDim.x * blockDim.x) {
        cnt[i] = 0;
        first[i] = INT_MAX;
    }
}

// per (block, tile row): how many kept points, and the first of them
__global__ void kept_count_kernel(KeptOrder o, const int* n_points, const int* point_tile, int* cnt, int* first)
{
    const int N = *n_points;
    const int ne = (N + o.stride - 1) / o.stride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        int block, row;
        kept_slot(o, point_tile[(size_t)e * o.stride], block, row);
        atomicAdd(cnt + block * o.sr + row, 1);
        atomicMin(first + block * o.sr + row, e);
    }
}

// exclusive scan of the per-slot counts in slot order (one block)
__global__ void __launch_bounds__(256) kept_scan_kernel(const int* cnt, int* offset, int n_slots)
{
    __shared__ int s_part[256];
    const int per = (n_slots + 255) / 256;
    const int beg = min(n_slots, (int)threadIdx.x * per), end = min(n_slots, beg + per);
    int sum = 0;
    for (int i = beg; i < end; ++i) sum += cnt[i];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < 256; ++t) {
            const int v = s_part[t];
            s_part[t] = acc;
            acc += v;
        }
    }
    __syncthreads();
    int acc = s_part[threadIdx.x];
    for (int i = beg; i < end; ++i) {
        offset[i] = acc;
        acc += cnt[i];
    }
}

__global__ void kept_write_kernel(KeptOrder o, const int* n_points, const float4* __restrict__ pts,
                                  const int* point_tile, const int* first, const int* offset, float4* kept,
                                  int* kept_count)
{
    const int N = *n_points;
    const int ne = (N + o.stride - 1) / o.stride;
    if (blockIdx.x == 0 && threadIdx.x == 0) *kept_count = ne;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        int block, row;
        const size_t j = (size_t)e * o.stride;
        kept_slot(o, point_tile[j], block, row);
        const int slot = block * o.sr + row;
        kept[offset[slot] + (e - first[slot])] = pts[j];
    }
}

// number of back-projection blocks for a w x h image
int bp_blocks(int width, int height)
{
    const int n_tiles = ((width + TILE_W - 1) / TILE_W) * ((height + TILE_H - 1) / TILE_H);
    return (n_tiles + BP_CHUNK_TILES - 1) / BP_CHUNK_TILES;
}

// ---------------------------------------------------------------------------
// Fitness
// ---------------------------------------------------------------------------
constexpr int FIT_THREADS = 256;
constexpr int FIT_WARPS = FIT_THREADS / 32;
constexpr int KC = 32;    // particles per CTA
constexpr int PPT = 4;    // points per thread per sub-tile
constexpr int SUBTILE = FIT_THREADS * PPT;

enum Source { SRC_POSES = 0, SRC_SEARCH = 1, SRC_EVAL = 2 };

struct FitArgs {
    const float4* pts;
    const int* n_dev;     // device point count, or nullptr to use n_host
    int n_host;
    int stride;           // evaluate points 0, stride, 2*stride, ...
    int K;                // particles of this launch
    const float* poses;   // SRC_POSES: K x 12
    float pm_threshold;   // particles on lanes when the chunk's spread (voxels) is below this
    const float* templ;   // SRC_SEARCH: templates, row k = particle k
    const void* chunks;   // the launch's particle chunks built by chunk_build_kernel, or null: each CTA builds its own
    // search, two-level reduction (or null: the launch's last CTA reduces
    // every particle over the point tiles): the last CTA of each chunk writes
    // its particles' E and count here, the last chunk to finish selects
    unsigned int* chunk_counter;
    float* chunk_E;
    int* chunk_C;
    SearchState* st;
    int compose_mode, update_mode;
    double beta;
    float min_valid_frac;
    // volume
    const void* tsdf;
    const void* weight;
    const void* cells;
    const float* cells32; // 16-/8-bit grids, full view: the records as floats too (else null)
    int nx, ny, nz;
    double vs;
    double org[3];
    // reduction
    float* part_S;
    int* part_C;
    unsigned int* counter;
    int n_ptiles;
    // outputs
    float* out_E;
    int* out_C;
    pf_track_stats* stats;
    int iter;
};

// Rodrigues' formula R = I + a [w]x + b [w]x^2 with a = sin(th)/th and
// b = (1 - cos th)/th^2, th = |w|.  SERIES (the chunk build's form): up to
// th = 1 rad both come from their Taylor series in th^2 (a = sum (-th^2)^n /
// (2n+1)!, b = sum (-th^2)^n / (2n+2)!, nine terms each: the first omitted
// term is below 1e-17, and both agree with the closed form to ~1e-16
// relative), which needs no square root, division or trigonometric call:
// the search's rotations are a few degrees, and the FP64 chain of each
// particle's construction is that kernel's latency.  Otherwise the closed
// form (its first terms below th = 1e-8).
template <bool SERIES = false>
__device__ inline void so3_exp_d(const double w[3], double R[9])
{
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double a, b;
    if (SERIES && th2 <= 1.0) {
        const double ca[9] = {1.0, -0.16666666666666666, 0.008333333333333333, -0.0001984126984126984,
                              2.7557319223985893e-06, -2.505210838544172e-08, 1.6059043836821613e-10,
                              -7.647163731819816e-13, 2.8114572543455206e-15};  // (-1)^n / (2n+1)!
        const double cb[9] = {0.5, -0.041666666666666664, 0.001388888888888889, -2.48015873015873e-05,
                              2.755731922398589e-07, -2.08767569878681e-09, 1.1470745597729725e-11,
                              -4.779477332387385e-14, 1.5619206968586225e-16};  // (-1)^n / (2n+2)!
        a = ca[8];
        b = cb[8];
        for (int n = 7; n >= 0; --n) {
            a = fma(a, th2, ca[n]);
            b = fma(b, th2, cb[n]);
        }
    } else {
        const double th = sqrt(th2);
        if (th < 1e-8) {
            a = 1.0 - th2 / 6.0;
            b = 0.5 - th2 / 24.0;
        } else {
            double sh = sin(0.5 * th), ch = cos(0.5 * th);
            a = 2.0 * sh * ch / th;
            b = 2.0 * sh * sh / th2;
        }
    }
    R[0] = 1.0 - b * (w[1] * w[1] + w[2] * w[2]);
    R[1] = -a * w[2] + b * w[0] * w[1];
    R[2] = a * w[1] + b * w[0] * w[2];
    R[3] = a * w[2] + b * w[0] * w[1];
    R[4] = 1.0 - b * (w[0] * w[0] + w[2] * w[2]);
    R[5] = -a * w[0] + b * w[1] * w[2];
    R[6] = -a * w[1] + b * w[0] * w[2];
    R[7] = a * w[0] + b * w[1] * w[2];
    R[8] = 1.0 - b * (w[0] * w[0] + w[1] * w[1]);
}

// Pose update in FP64: out = [dR | dt] applied to P (mode 0: dR*R, dR*t+dt;
// mode 1: dR*R, t+dt), then one Newton-Schulz step R <- R (3I - R^T R)/2
// to restore orthonormality.
__device__ inline void compose_d(const double dR[9], const double dt[3], const double P[12], int mode,
                                 double out[12])
{
    double R[9];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            R[3 * r + c] = dR[3 * r] * P[c] + dR[3 * r + 1] * P[4 + c] + dR[3 * r + 2] * P[8 + c];
        const double tr = mode == 0 ? dR[3 * r] * P[3] + dR[3 * r + 1] * P[7] + dR[3 * r + 2] * P[11] : P[4 * r + 3];
        out[4 * r + 3] = tr + dt[r];
    }
    double M[9];  // R^T R
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[r] * R[c] + R[3 + r] * R[3 + c] + R[6 + r] * R[6 + c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += R[3 * r + m] * ((m == c ? 3.0 : 0.0) - M[3 * m + c]);
            out[4 * r + c] = 0.5 * acc;
        }
}

// Particles as the sampling loop uses them.
//
// Particle k maps a camera-frame point x to grid units, relative to an
// integer cell offset o_k, as g_k = A_k x + b_k with A_k = R_k / voxel and
// b_k = (t_k - origin) / voxel - o_k in [0, 1).  The CTA splits
// A_k = A_ref + dA_k, where A_ref is its first particle's matrix carried as a
// float pair (hi + lo): y = A_ref x is formed once per point and shared by
// all particles of the chunk, and each sample adds dA_k x + b_k in float.
// dA_k is small (the particles of a chunk differ by the search size), so its
// float rounding is negligible, and every sample position is as accurate as
// the FP64 pose it came from; rounding a whole float matrix per particle
// would instead shift all points of that particle alike.  The offset o_k is
// folded into the magic constant of the floor and costs nothing per sample.
struct Particle {      // shared memory, 64 bytes
    float4 d0, d1, d2; // rows of dA_k | b_k
    int4 m;            // magic x, y, z (cell offset folded in), unused
};

constexpr int kMagicBits = 0x4b400000;  // bits of 1.5 * 2^23
constexpr int kNeverValid = 0x7fffffff;  // magic of a particle that reaches no cell

// Camera-to-world pose of particle k in FP64.
template <int SRC, bool SERIES = false>
__device__ inline void particle_pose(const FitArgs& a, int k, double R[9], double tw[3])
{
    if (SRC == SRC_POSES) {
        const float* p = a.poses + 12 * (size_t)k;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) R[3 * r + c] = (double)p[4 * r + c];
            tw[r] = (double)p[4 * r + 3];
        }
    } else {
        const double* P = a.st->P;
        if (SRC == SRC_EVAL) {
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c) R[3 * r + c] = P[4 * r + c];
                tw[r] = P[4 * r + 3];
            }
        } else {
            const float* u = a.templ + 6 * (size_t)k;
            const double wr = a.st->s[0] * kPi / 180.0, wt = a.st->s[1] / 100.0;
            const double dw[3] = {wr * (double)u[0], wr * (double)u[1], wr * (double)u[2]};
            double dR[9];
            so3_exp_d<SERIES>(dw, dR);
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c)
                    R[3 * r + c] = dR[3 * r] * P[c] + dR[3 * r + 1] * P[4 + c] + dR[3 * r + 2] * P[8 + c];
                const double tr = a.compose_mode == 0 ? dR[3 * r] * P[3] + dR[3 * r + 1] * P[7] + dR[3 * r + 2] * P[11]
                                                      : P[4 * r + 3];
                tw[r] = tr + wt * (double)u[3 + r];
            }
        }
    }
}

// A particle as the plain float form uses it: grid coordinate = A x + c,
// A = R / vs, c = (t - origin) / vs, both rounded to float.
struct PlainXf {
    float A[9];
    float c[3];
};

// Particles k_begin .. k_begin+kc-1 into shared memory, and the chunk's
// reference matrix A_ref (its first particle) as hi and lo floats; with
// sAbs, also each particle's plain float transform.
// CHUNK (the chunk build kernel): the series form of the exponential, and
// thread 0's pose (the chunk's first particle) passed to the other threads
// by shuffles instead of each thread forming it again.
template <int SRC, bool CHUNK = false>
__device__ void build_particles(const FitArgs& a, int k_begin, int kc, Particle* sP, float* sRef, PlainXf* sAbs)
{
    const int t = threadIdx.x;  // (kc <= KC = 32: one warp)
    if (t >= kc) return;
    double R[9], tw[3], R0[9], t0[3];
    particle_pose<SRC, CHUNK>(a, k_begin + t, R, tw);
    if (CHUNK) {
        const unsigned lanes = kc >= 32 ? 0xffffffffu : (1u << kc) - 1u;
        for (int q = 0; q < 9; ++q) R0[q] = __shfl_sync(lanes, R[q], 0);
        for (int r = 0; r < 3; ++r) t0[r] = __shfl_sync(lanes, tw[r], 0);
    } else {
        particle_pose<SRC>(a, k_begin, R0, t0);
    }
    const double iv = 1.0 / a.vs;
    float d[9], b[3];
    int magic[3];
    bool ok = true;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) d[3 * r + c] = (float)(R[3 * r + c] * iv - R0[3 * r + c] * iv);
        const double tg = (tw[r] - a.org[r]) * iv;
        ok = ok && fabs(tg) < 2097152.0;  // 2^21: beyond, no point can reach the grid
        const double o = ok ? floor(tg) : 0.0;
        b[r] = (float)(tg - o);
        magic[r] = kMagicBits - (int)o;
    }
    if (!ok) magic[0] = kNeverValid;
    if (sAbs) {
        for (int q = 0; q < 9; ++q) sAbs[t].A[q] = (float)(R[q] * iv);
        for (int r = 0; r < 3; ++r) sAbs[t].c[r] = (float)((tw[r] - a.org[r]) * iv);
    }
    sP[t].d0 = make_float4(d[0], d[1], d[2], b[0]);
    sP[t].d1 = make_float4(d[3], d[4], d[5], b[1]);
    sP[t].d2 = make_float4(d[6], d[7], d[8], b[2]);
    sP[t].m = make_int4(magic[0], magic[1], magic[2], 0);
    if (t == 0)
        for (int q = 0; q < 9; ++q) {
            const double A0 = R0[q] * iv;
            const float hi = (float)A0;
            sRef[q] = hi;
            sRef[9 + q] = (float)(A0 - (double)hi);
        }
}

// One row of y = A_ref x, with A_ref = hi + lo, accurate to ~1e-12 of |y|
// (exact products and two-sums in float), returned as an integer part and a
// fraction: y = yi + yf with |yf| <= ~0.5.  Done once per point per block of
// points and shared by every particle of the chunk, so each sample only
// rounds at the scale of dA_k x + yf + b_k (a few voxels) rather than at the
// scale of the grid coordinate itself.
__device__ __forceinline__ void ref_row(const float* hi, const float* lo, float x, float y, float z, int& yi, float& yf)
{
    const float p0 = hi[0] * x, p1 = hi[1] * y, p2 = hi[2] * z;
    float err = fmaf(hi[0], x, -p0) + fmaf(hi[1], y, -p1) + fmaf(hi[2], z, -p2);
    const float s1 = p0 + p1;
    float bb = s1 - p0;
    err += (p0 - (s1 - bb)) + (p1 - bb);
    const float s2 = s1 + p2;
    bb = s2 - s1;
    err += (s1 - (s2 - bb)) + (p2 - bb);
    err = fmaf(lo[0], x, fmaf(lo[1], y, fmaf(lo[2], z, err)));
    const float r = rintf(s2);
    yi = __float2int_rn(r);
    yf = (s2 - r) + err;
}

__device__ __forceinline__ void ref_apply(const float* Rf, float x, float y, float z, int* Yi, float* Yf)
{
    ref_row(Rf + 0, Rf + 9, x, y, z, Yi[0], Yf[0]);
    ref_row(Rf + 3, Rf + 12, x, y, z, Yi[1], Yf[1]);
    ref_row(Rf + 6, Rf + 15, x, y, z, Yi[2], Yf[2]);
}

// Grid cell of a sample and its fractions.  The grid coordinate is
// o_k + yi + (dA_k x + yf + b_k); the bracket is small and its floor comes
// from adding 1.5*2^23 rounding down, which leaves floor() in the low
// mantissa bits with every step exact (for |.| < 2^22).  Subtracting the
// particle's magic constant adds o_k, and yi is added in the same integer
// instruction.  Any coordinate outside [0, n-1), including NaN, gives an
// index outside that range on some axis (huge values wrap far outside), so
// one unsigned compare per axis is the whole range test.
struct Cell {
    int idx;
    float fx, fy, fz;
    bool ok;
};

__device__ __forceinline__ void accumulate(float t, float& s, int& c)
{
    t = fabsf(t);
    if (t < INFINITY) {  // non-finite: some corner unobserved or outside the band
        s += t;
        c += 1;
    }
}

// Trilinear interpolation from a cell-view record: corners with their
// x-differences already formed (v000, v100 - v000, v010, v110 - v010, ...).
// (A packed f32x2 form of these steps was measured slower: it needs the
// fractions duplicated into register pairs.)
__device__ __forceinline__ float trilerp_cell(float fx, float fy, float fz, float4 lo, float4 hi)
{
    const float x00 = fmaf(fx, lo.y, lo.x);
    const float x10 = fmaf(fx, lo.w, lo.z);
    const float x01 = fmaf(fx, hi.y, hi.x);
    const float x11 = fmaf(fx, hi.w, hi.z);
    const float y0 = fmaf(fy, x10 - x00, x00);
    const float y1 = fmaf(fy, x11 - x01, x01);
    return fmaf(fz, y1 - y0, y0);
}

__device__ __forceinline__ float trilerp(float fx, float fy, float fz, float v000, float v100, float v010, float v110,
                                         float v001, float v101, float v011, float v111)
{
    const float x00 = fmaf(fx, v100 - v000, v000);
    const float x10 = fmaf(fx, v110 - v010, v010);
    const float x01 = fmaf(fx, v101 - v001, v001);
    const float x11 = fmaf(fx, v111 - v011, v011);
    const float y0 = fmaf(fy, x10 - x00, x00);
    const float y1 = fmaf(fy, x11 - x01, x01);
    return fmaf(fz, y1 - y0, y0);
}

// A cell-view record as two float4: (v000, v100 - v000, v010, v110 - v010)
// and (v001, v101 - v001, v011, v111 - v011).  Float storage keeps that form
// (two 16-byte loads of one sector); half / bfloat16 storage keeps the eight
// corners as stored (one 16-byte load) and the differences are formed here.
__device__ __forceinline__ void load_cell(const float* cells, int idx, float4& lo, float4& hi)
{
    // one 32-byte record, one 256-bit read-only load (records are 32-byte
    // aligned): half the load requests of two 16-byte loads.  volatile: the
    // load must not be hoisted above the range test that guards it.
    const float* p = cells + 8 * (size_t)idx;
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(p));
}

__device__ __forceinline__ void corners_to_cell(float v000, float v100, float v010, float v110, float v001,
                                                float v101, float v011, float v111, float4& lo, float4& hi)
{
    lo = make_float4(v000, v100 - v000, v010, v110 - v010);
    hi = make_float4(v001, v101 - v001, v011, v111 - v011);
}

__device__ __forceinline__ void load_cell(const __half* cells, int idx, float4& lo, float4& hi)
{
    const uint4 r = __ldg(reinterpret_cast<const uint4*>(cells) + idx);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    const float2 c = __half22float2(*reinterpret_cast<const __half2*>(&r.z));
    const float2 d = __half22float2(*reinterpret_cast<const __half2*>(&r.w));
    corners_to_cell(a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y, lo, hi);
}

// Scaled e4m3 records: one 8-byte load; each pair of codes goes to half2 in
// one conversion and is multiplied by 160 in half, which is exact (3 + 3
// significant bits) for every value code and overflows the outside-the-band
// code 448 to infinity (448 x 160 > 65504 > 240 x 160), so the float record
// below holds 160 x 256 = 40960 times the stored values, with the band's
// edge non-finite as in the other layouts; the interpolated value is scaled
// back once (cell_scale).
__device__ __forceinline__ void load_cell(const __nv_fp8_e4m3* cells, int idx, float4& lo, float4& hi)
{
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(cells) + idx);
    const __half2 k = __floats2half2_rn(160.0f, 160.0f);
    float2 q[4];
    const unsigned short pairs[4] = {(unsigned short)(r.x & 0xffffu), (unsigned short)(r.x >> 16),
                                     (unsigned short)(r.y & 0xffffu), (unsigned short)(r.y >> 16)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2 h(__nv_cvt_fp8x2_to_halfraw2(pairs[i], __NV_E4M3));
        q[i] = __half22float2(__hmul2(h, k));
    }
    corners_to_cell(q[0].x, q[0].y, q[1].x, q[1].y, q[2].x, q[2].y, q[3].x, q[3].y, lo, hi);
}

template <typename T>
__device__ __forceinline__ constexpr float cell_scale()
{
    return std::is_same<T, __nv_fp8_e4m3>::value ? 1.0f / (160.0f * PF_FP8_SCALE) : 1.0f;
}

__device__ __forceinline__ void load_cell(const __nv_bfloat16* cells, int idx, float4& lo, float4& hi)
{
    // a bfloat16 is the upper half of a float
    const uint4 r = __ldg(reinterpret_cast<const uint4*>(cells) + idx);
    corners_to_cell(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                    __uint_as_float(r.y & 0xffff0000u), __uint_as_float(r.z << 16), __uint_as_float(r.z & 0xffff0000u),
                    __uint_as_float(r.w << 16), __uint_as_float(r.w & 0xffff0000u), lo, hi);
}

// Gather and accumulate one located sample.  VARIANT 0: encoded tsdf nodes (non-finite nodes make the
// interpolated value non-finite, so validity is one comparison on the
// result); 1: plain tsdf + weight (float), all eight nodes tested
// explicitly; 2: the cell view.  TS is the storage type of tsdf and cells.
// BRANCHLESS (cell view only): a sample outside the grid reads cell 0 and is
// dropped by the final predicate instead of a branch -- cheaper when almost
// every sample lands inside, as when particles share the lanes of a warp.
template <int VARIANT, typename TS, bool BRANCHLESS = false, bool FLOAT_CELLS = false>
__device__ __forceinline__ void gather(const FitArgs& a, int nx, int nxy, const Cell& q, float& s, int& c)
{
    if (VARIANT == 2 && BRANCHLESS) {
        float4 lo, hi;
        if (FLOAT_CELLS)
            load_cell(a.cells32, q.ok ? q.idx : 0, lo, hi);
        else
            load_cell(static_cast<const TS*>(a.cells), q.ok ? q.idx : 0, lo, hi);
        constexpr float k = FLOAT_CELLS ? 1.0f : cell_scale<TS>();
        const float t = fabsf(trilerp_cell(q.fx, q.fy, q.fz, lo, hi)) * k;
        const bool use = q.ok && t < INFINITY;
        s += use ? t : 0.0f;
        c += use ? 1 : 0;
        return;
    }
    if (!q.ok) return;
    if (VARIANT == 2) {
        float4 lo, hi;
        load_cell(static_cast<const TS*>(a.cells), q.idx, lo, hi);
        accumulate(trilerp_cell(q.fx, q.fy, q.fz, lo, hi) * cell_scale<TS>(), s, c);
    } else if (VARIANT == 0) {
        const TS* p = static_cast<const TS*>(a.tsdf) + q.idx;
        accumulate(trilerp(q.fx, q.fy, q.fz, pf_to_float(p[0]), pf_to_float(p[1]), pf_to_float(p[nx]),
                           pf_to_float(p[nx + 1]), pf_to_float(p[nxy]), pf_to_float(p[nxy + 1]),
                           pf_to_float(p[nxy + nx]), pf_to_float(p[nxy + nx + 1])),
                   s, c);
    } else {
        const float* tsdf = static_cast<const float*>(a.tsdf);
        const float* weight = static_cast<const float*>(a.weight);
        const int off[8] = {0, 1, nx, nx + 1, nxy, nxy + 1, nxy + nx, nxy + nx + 1};
        float v[8];
        bool ok = true;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float w = __ldg(weight + q.idx + off[r]);
            v[r] = __ldg(tsdf + q.idx + off[r]);
            ok = ok && (w > 0.0f) && (fabsf(v[r]) < 1.0f);
        }
        if (ok) {
            s += fabsf(trilerp(q.fx, q.fy, q.fz, v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]));
            c += 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Two samples at once.  Blackwell's packed f32x2 FMA / add instructions do
// two float operations per instruction with exactly the rounding of two
// scalar ones, so the transform, the floor and the fractions of two samples
// cost half the issue slots and give bit-identical results.  The pair is two
// points of one particle; the particle's values are held duplicated.
// ---------------------------------------------------------------------------
struct ParticleD {     // shared memory, 112 bytes
    float4 d[6];       // (d0, d0, d1, d1), (d2, d2, d3, d3), ..., (d8, d8, b0, b0), (b1, b1, b2, b2)
    int4 m;            // magic x, y, z and cl = -(mx + nx my + nxy mz) (wrapping)
};

struct XformD {
    float2 d[9], b[3];
    int mg[3];
    int cl;
};

__device__ __forceinline__ void make_particle_d(const Particle& P, int nx, int nxy, ParticleD& D)
{
    const float v[12] = {P.d0.x, P.d0.y, P.d0.z, P.d1.x, P.d1.y, P.d1.z,
                         P.d2.x, P.d2.y, P.d2.z, P.d0.w, P.d1.w, P.d2.w};
    for (int q = 0; q < 6; ++q) D.d[q] = make_float4(v[2 * q], v[2 * q], v[2 * q + 1], v[2 * q + 1]);
    const unsigned cl = 0u - ((unsigned)P.m.x + (unsigned)nx * (unsigned)P.m.y + (unsigned)nxy * (unsigned)P.m.z);
    D.m = make_int4(P.m.x, P.m.y, P.m.z, (int)cl);
}

__device__ __forceinline__ void load_xformd(const ParticleD& P, XformD& X)
{
    float2 v[12];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 f = P.d[q];
        v[2 * q] = make_float2(f.x, f.y);
        v[2 * q + 1] = make_float2(f.z, f.w);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) X.d[q] = v[q];
    X.b[0] = v[9];
    X.b[1] = v[10];
    X.b[2] = v[11];
    X.mg[0] = P.m.x;
    X.mg[1] = P.m.y;
    X.mg[2] = P.m.z;
    X.cl = P.m.w;
}

// Two points (a, b) of the same sub-tile: coordinates and reference
// fractions as pairs, and the linear index of each reference cell,
// yl = yi_x + nx yi_y + nxy yi_z.
struct PointPair {
    float2 x, y, z, yf0, yf1, yf2;
    int yla, ylb;
};

// Cells and fractions of a pair of samples.  The packed part (transform,
// floor, fractions) follows the grid-cell rule above for two points.  CHECKED = false:
// the caller knows both cells lie inside the grid (the points passed the
// chunk's interior test), so there is no range test and the cell index is
// one linear combination, idx = yl + cl + bits(rx) + nx bits(ry) +
// nxy bits(rz) -- the value of the per-axis form (wrapping arithmetic, exact
// result in range).  CHECKED = true: per-axis cells from the reference cells
// Ya, Yb and the unsigned range test.
template <bool CHECKED>
__device__ __forceinline__ void locate2(const XformD& X, int nx, int nxy, unsigned mx, unsigned my, unsigned mz,
                                        const PointPair& p, const int* Ya, const int* Yb, Cell& ca, Cell& cb)
{
    const float2 gx = __ffma2_rn(X.d[0], p.x, __ffma2_rn(X.d[1], p.y, __ffma2_rn(X.d[2], p.z, __fadd2_rn(p.yf0, X.b[0]))));
    const float2 gy = __ffma2_rn(X.d[3], p.x, __ffma2_rn(X.d[4], p.y, __ffma2_rn(X.d[5], p.z, __fadd2_rn(p.yf1, X.b[1]))));
    const float2 gz = __ffma2_rn(X.d[6], p.x, __ffma2_rn(X.d[7], p.y, __ffma2_rn(X.d[8], p.z, __fadd2_rn(p.yf2, X.b[2]))));
    const float2 M2 = make_float2(12582912.0f, 12582912.0f), nM2 = make_float2(-12582912.0f, -12582912.0f);
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 rx = __fadd2_rd(gx, M2), ry = __fadd2_rd(gy, M2), rz = __fadd2_rd(gz, M2);
    // g - (r - M): r - M is exact, and -1 * t + g rounds once like g - t
    const float2 fx = __ffma2_rn(__fadd2_rn(rx, nM2), m1, gx);
    const float2 fy = __ffma2_rn(__fadd2_rn(ry, nM2), m1, gy);
    const float2 fz = __ffma2_rn(__fadd2_rn(rz, nM2), m1, gz);
    if (CHECKED) {
        const int ax = __float_as_int(rx.x) - X.mg[0] + Ya[0], bx = __float_as_int(rx.y) - X.mg[0] + Yb[0];
        const int ay = __float_as_int(ry.x) - X.mg[1] + Ya[1], by = __float_as_int(ry.y) - X.mg[1] + Yb[1];
        const int az = __float_as_int(rz.x) - X.mg[2] + Ya[2], bz = __float_as_int(rz.y) - X.mg[2] + Yb[2];
        ca.ok = (unsigned)ax < mx && (unsigned)ay < my && (unsigned)az < mz;
        cb.ok = (unsigned)bx < mx && (unsigned)by < my && (unsigned)bz < mz;
        ca.idx = ax + nx * ay + nxy * az;
        cb.idx = bx + nx * by + nxy * bz;
    } else {
        const unsigned ux = (unsigned)nx, uxy = (unsigned)nxy;
        ca.idx = (int)((unsigned)p.yla + (unsigned)X.cl + (unsigned)__float_as_int(rx.x) +
                       ux * (unsigned)__float_as_int(ry.x) + uxy * (unsigned)__float_as_int(rz.x));
        cb.idx = (int)((unsigned)p.ylb + (unsigned)X.cl + (unsigned)__float_as_int(rx.y) +
                       ux * (unsigned)__float_as_int(ry.y) + uxy * (unsigned)__float_as_int(rz.y));
        ca.ok = true;
        cb.ok = true;
    }
    ca.fx = fx.x; ca.fy = fy.x; ca.fz = fz.x;
    cb.fx = fx.y; cb.fy = fy.y; cb.fz = fz.y;
}

// Whether every sample of point (Yi, Yf) under any particle of the chunk
// lands in a cell inside the grid: lo[a] <= yi_a <= hi[a] on every axis
// (bounds from the chunk's reach, see the kernel) and a finite point.
__device__ __forceinline__ bool point_interior(const int* Yi, const float* Yf, const int* lo, const int* hi)
{
    bool in = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) in = in && Yi[q] >= lo[q] && Yi[q] <= hi[q] && fabsf(Yf[q]) <= 1.0f;
    return in;
}

__device__ __forceinline__ int linear_cell(const int* Yi, int nx, int nxy)
{
    return (int)((unsigned)Yi[0] + (unsigned)nx * (unsigned)Yi[1] + (unsigned)nxy * (unsigned)Yi[2]);
}

// Block-wide argmin of (E, k) with the lowest k among equal E.
__device__ inline void argmin_pair(float& e, int& k, float* se, int* sk)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
        const int k2 = __shfl_xor_sync(0xffffffffu, k, o);
        if (e2 < e || (e2 == e && k2 < k)) {
            e = e2;
            k = k2;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        se[warp] = e;
        sk[warp] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < FIT_WARPS; ++w)
            if (se[w] < se[0] || (se[w] == se[0] && sk[w] < sk[0])) {
                se[0] = se[w];
                sk[0] = sk[w];
            }
    }
    __syncthreads();
    e = se[0];
    k = sk[0];
    __syncthreads();
}

#ifndef PF_FIT_MIN_BLOCKS
#define PF_FIT_MIN_BLOCKS 3
#endif

// Sums of one particle's partials over the point tiles, S = sum of
// part_S[y K + k] and C likewise for y = 0, 1, ..., T - 1 in that order.
// The loads go out 16 at a time before they are added (in the same order),
// so the last CTA waits one L2 round trip per 16 tiles instead of a few per
// tile.  Adding 0 for the padding slots leaves the float sum unchanged (the
// partial sums are non-negative), so the result is that of the plain loop.
__device__ __forceinline__ void sum_tiles(const float* part_S, const int* part_C, int K, int T, int k, float& S,
                                          int& C)
{
    constexpr int B = 16;
    S = 0.0f;
    C = 0;
    for (int y0 = 0; y0 < T; y0 += B) {
        float sv[B];
        int cv[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const bool in = y0 + q < T;
            const size_t o = (size_t)(in ? y0 + q : y0) * K + k;
            sv[q] = in ? __ldcg(part_S + o) : 0.0f;
            cv[q] = in ? __ldcg(part_C + o) : 0;
        }
#pragma unroll
        for (int q = 0; q < B; ++q) {
            S += sv[q];
            C += cv[q];
        }
    }
}

// A particle chunk as a fitness CTA uses it: the chunk's particles in both
// forms, its reference matrix as a float pair, and the chunk's spread and
// reach (see fitness_body).  chunk_build_kernel forms it once per search
// iteration, one warp per chunk, so the CTAs of the chunk's point tiles copy
// it instead of each repeating the FP64 construction of 32 particles (~20 us
// per CTA, measured) and the serial reach loop.
struct ChunkData {
    Particle P[KC];
    ParticleD PD[KC];
    float ref[18];
    float spread[2];   // largest translation (voxels) and rotation (voxels per metre) against particle 0
    float dmax;        // largest row sum of |dA_k| (infinite when some particle is not finite)
    int omin[3], omax[3];
    int pad;
};
static_assert(sizeof(ChunkData) % 16 == 0, "ChunkData is copied as 16-byte words");

// One warp per chunk: thread t builds particle k_begin + t exactly as a CTA
// would (build_particles, make_particle_d), and the chunk's spread and reach
// come from warp reductions of the per-particle values (maxima and minima:
// the same values as the serial loop, whatever the order).
template <int SRC>
__global__ void __launch_bounds__(32) chunk_build_kernel(FitArgs a, ChunkData* out)
{
    const int t = threadIdx.x;
    const int k_begin = blockIdx.x * KC;
    const int kc = min(KC, a.K - k_begin);
    if (SRC != SRC_POSES && a.st->lost) return;  // the fitness launch skips every chunk then
    ChunkData& C = out[blockIdx.x];
    const int nx = a.nx, nxy = a.nx * a.ny;
    build_particles<SRC, true>(a, k_begin, kc, C.P, C.ref, nullptr);
    __syncwarp();
    const bool mine = t < kc;
    Particle P;
    if (mine) {
        P = C.P[t];
        make_particle_d(P, nx, nxy, C.PD[t]);
    }
    const float4 row[3] = {mine ? P.d0 : make_float4(0, 0, 0, 0), mine ? P.d1 : make_float4(0, 0, 0, 0),
                           mine ? P.d2 : make_float4(0, 0, 0, 0)};
    const int m[3] = {mine ? P.m.x : 0, mine ? P.m.y : 0, mine ? P.m.z : 0};
    float dt = 0.0f, dr = 0.0f, dmax = 0.0f;
    int omin[3], omax[3];
    for (int r = 0; r < 3; ++r) {
        // particle 0 of the chunk, as the serial loop takes it
        const float o0 = (float)(kMagicBits - __shfl_sync(0xffffffffu, m[r], 0));
        const float b0 = __shfl_sync(0xffffffffu, row[r].w, 0);
        const int o = kMagicBits - m[r];
        omin[r] = mine ? o : INT_MAX;
        omax[r] = mine ? o : INT_MIN;
        if (mine) {
            const float sum = fabsf(row[r].x) + fabsf(row[r].y) + fabsf(row[r].z);
            dmax = (sum < INFINITY && fabsf(row[r].w) <= 1.0f) ? fmaxf(dmax, sum) : INFINITY;
            if (t > 0) {
                dt = fmaxf(dt, fabsf((float)(kMagicBits - m[r]) + row[r].w - (o0 + b0)));
                dr = fmaxf(dr, sum);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        dt = fmaxf(dt, __shfl_xor_sync(0xffffffffu, dt, o));
        dr = fmaxf(dr, __shfl_xor_sync(0xffffffffu, dr, o));
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    }
    for (int r = 0; r < 3; ++r) {
        omin[r] = __reduce_min_sync(0xffffffffu, omin[r]);
        omax[r] = __reduce_max_sync(0xffffffffu, omax[r]);
    }
    if (t == 0) {
        C.spread[0] = dt;
        C.spread[1] = dr;
        C.dmax = dmax;
        for (int r = 0; r < 3; ++r) {
            C.omin[r] = omin[r];
            C.omax[r] = omax[r];
        }
        C.pad = 0;
    }
}

// The work of one CTA: particle chunk bx, point tile by, of a launch of
// n_blocks CTAs for this problem (the last of them to finish runs the
// epilogue).
// SOLO: a launch of one problem, which may use prebuilt particle chunks and
// the two-level reduction (FitArgs.chunks, .chunk_counter); the batched
// launch compiles without them.
template <int SRC, int VARIANT, typename TS, bool SOLO>
__device__ __forceinline__ void fitness_body(const FitArgs& a, int bx, int by, unsigned n_blocks)
{
    __shared__ __align__(16) ChunkData sC;
    Particle* const sP = sC.P;
    ParticleD* const sPD = sC.PD;
    float* const sRef = sC.ref;
    __shared__ PlainXf sAbs[VARIANT == 1 ? KC : 1];
    // particles on lanes: each warp's points as pairs (point q, point q + 64
    // of the warp): (x, y), (z, yf0), (yf1, yf2), and their reference cells
    __shared__ float4 sPair[FIT_WARPS][PPT * 16][3];
    __shared__ int2 sPyl[FIT_WARPS][PPT * 16];
    __shared__ float accS[FIT_WARPS][KC];
    __shared__ int accC[FIT_WARPS][KC];
    __shared__ int s_last;
    __shared__ int s_skip;
    __shared__ int s_mode;
    float* const s_spread = sC.spread;
    __shared__ float s_red[FIT_WARPS];
    float& s_dmax = sC.dmax;
    __shared__ long long s_omin[3], s_omax[3];
    __shared__ int s_lo[3], s_hi[3];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k_begin = bx * KC;
    const int kc = min(KC, a.K - k_begin);
    const int nx = a.nx, nxy = a.nx * a.ny;
    const unsigned mx = a.nx - 1, my = a.ny - 1, mz = a.nz - 1;

    if (tid == 0) {
        int skip = 0;
        if (SRC != SRC_POSES) {
            skip = a.st->lost;
            if (SRC == SRC_EVAL) skip = skip || !a.st->pending_s;
        }
        s_skip = skip;
    }
    for (int q = tid; q < FIT_WARPS * KC; q += FIT_THREADS) {
        (&accS[0][0])[q] = 0.0f;
        (&accC[0][0])[q] = 0;
    }
    __syncthreads();
    const bool skip = s_skip != 0;
    const bool prebuilt = SOLO && SRC == SRC_SEARCH && a.chunks != nullptr;  // (never with the plain layout)
    if (!skip) {
        if (prebuilt) {
            const int4* src = reinterpret_cast<const int4*>(static_cast<const ChunkData*>(a.chunks) + bx);
            int4* dst = reinterpret_cast<int4*>(&sC);
            for (int q = tid; q < (int)(sizeof(ChunkData) / 16); q += FIT_THREADS) dst[q] = __ldg(src + q);
        } else {
            build_particles<SRC>(a, k_begin, kc, sP, sRef, VARIANT == 1 ? sAbs : nullptr);
            if (tid < kc) make_particle_d(sP[tid], nx, nxy, sPD[tid]);
        }
    }
    __syncthreads();
    if (prebuilt && tid == 0) {
        for (int r = 0; r < 3; ++r) {
            s_omin[r] = skip ? LLONG_MAX : (long long)sC.omin[r];
            s_omax[r] = skip ? LLONG_MIN : (long long)sC.omax[r];
        }
    }
    // spread of the chunk's particles relative to its first one: translation
    // (voxels) and rotation (voxels per metre of point distance); and the
    // chunk's reach: the range of the particles' integer cell offsets o_k
    // and the largest row sum of |dA_k|, which bound where any particle can
    // put a point (see the interior test below)
    if (!prebuilt && tid == 0) {
        float dt = 0.0f, dr = 0.0f, dmax = 0.0f;
        long long omin[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, omax[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        if (!skip) {
            const float o0[3] = {(float)(kMagicBits - sP[0].m.x), (float)(kMagicBits - sP[0].m.y),
                                 (float)(kMagicBits - sP[0].m.z)};
            const float b0[3] = {sP[0].d0.w, sP[0].d1.w, sP[0].d2.w};
            for (int k = 0; k < kc; ++k) {
                const Particle& P = sP[k];
                const float4 row[3] = {P.d0, P.d1, P.d2};
                const int m[3] = {P.m.x, P.m.y, P.m.z};
                for (int r = 0; r < 3; ++r) {
                    const long long o = (long long)kMagicBits - (long long)m[r];
                    omin[r] = o < omin[r] ? o : omin[r];
                    omax[r] = o > omax[r] ? o : omax[r];
                    const float sum = fabsf(row[r].x) + fabsf(row[r].y) + fabsf(row[r].z);
                    // a non-finite particle disables the interior path
                    dmax = (sum < INFINITY && fabsf(row[r].w) <= 1.0f) ? fmaxf(dmax, sum) : INFINITY;
                    if (k > 0) {
                        dt = fmaxf(dt, fabsf((float)(kMagicBits - m[r]) + row[r].w - (o0[r] + b0[r])));
                        dr = fmaxf(dr, sum);
                    }
                }
            }
        }
        s_spread[0] = dt;
        s_spread[1] = dr;
        s_dmax = dmax;
        for (int r = 0; r < 3; ++r) {
            s_omin[r] = omin[r];
            s_omax[r] = omax[r];
        }
    }
    __syncthreads();

    const int N = a.n_dev ? *a.n_dev : a.n_host;
    const long long Ne = N > 0 ? ((long long)N + a.stride - 1) / a.stride : 0;
    const long long beg = Ne * by / a.n_ptiles;
    const long long end = Ne * (by + 1) / a.n_ptiles;

    if (!skip) {
        for (long long sub = beg; sub < end; sub += SUBTILE) {
            float px[PPT], py[PPT], pz[PPT];
            float r2 = 0.0f;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const long long e = sub + p * FIT_THREADS + tid;
                if (e < end) {
                    const float4 q = __ldg(a.pts + e * a.stride);
                    px[p] = q.x;
                    py[p] = q.y;
                    pz[p] = q.z;
                    r2 = fmaxf(r2, q.x * q.x + q.y * q.y + q.z * q.z);
                } else {
                    px[p] = NAN;
                    py[p] = NAN;
                    pz[p] = NAN;
                }
            }
            if (VARIANT == 1) {
                // The plain float form (the performance baseline): for each
                // particle, every point's grid coordinate A x + c in float,
                // floor, an explicit range test, eight tsdf and eight weight
                // loads; lanes on neighbouring points, warp-shuffle sums.
                for (int kk = 0; kk < kc; ++kk) {
                    const PlainXf& X = sAbs[kk];
                    float s = 0.0f;
                    int c = 0;
#pragma unroll
                    for (int p = 0; p < PPT; ++p) {
                        const float gx = fmaf(X.A[0], px[p], fmaf(X.A[1], py[p], fmaf(X.A[2], pz[p], X.c[0])));
                        const float gy = fmaf(X.A[3], px[p], fmaf(X.A[4], py[p], fmaf(X.A[5], pz[p], X.c[1])));
                        const float gz = fmaf(X.A[6], px[p], fmaf(X.A[7], py[p], fmaf(X.A[8], pz[p], X.c[2])));
                        if (!(gx >= 0.0f && gx < (float)(a.nx - 1) && gy >= 0.0f && gy < (float)(a.ny - 1) &&
                              gz >= 0.0f && gz < (float)(a.nz - 1)))
                            continue;
                        const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
                        Cell q;
                        q.idx = (int)fx0 + nx * (int)fy0 + nxy * (int)fz0;
                        q.fx = gx - fx0;
                        q.fy = gy - fy0;
                        q.fz = gz - fz0;
                        q.ok = true;
                        gather<1, float>(a, nx, nxy, q, s, c);
                    }
                    c = __reduce_add_sync(0xffffffffu, c);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) {
                        accS[warp][kk] += s;
                        accC[warp][kk] += c;
                    }
                }
                continue;
            }
            // mapping of this sub-tile: when every particle puts a point in
            // (nearly) the same cell, lanes take particles and share a point,
            // so each gather of a warp touches one or two sectors; otherwise
            // lanes take neighbouring image points of one particle
            // (the plain form never gets here: no unreachable-code note)
#pragma nv_diag_suppress 128
            for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
#pragma nv_diag_default 128
            if (lane == 0) s_red[warp] = r2;
            __syncthreads();
            if (tid == 0) {
                float m = 0.0f;
                for (int w = 0; w < FIT_WARPS; ++w) m = fmaxf(m, s_red[w]);
                const float rad = sqrtf(m);
                // (a chunk of fewer than 24 particles would leave lanes idle)
                s_mode = kc >= 24 && (s_spread[0] + s_spread[1] * rad) < a.pm_threshold;
                // Interior test.  Sample cell coordinate on axis r:
                // yi_r + o_k,r + floor(dA_k,r . x + yf_r + b_k,r) with
                // |yf| <= 1/2 + eps, 0 <= b < 1 and |dA_k,r . x| <= dmax |x|,
                // so it lies within yi_r + [omin_r - E, omax_r + E] for
                // E = ceil(dmax |x|) + 3 (one cell of margin).  A point whose
                // yi_r keeps that range inside [0, n_r - 2] on every axis
                // needs no range test under any particle of the chunk.
                const float reach = s_dmax * rad;
                const long long E = reach < 1.0e6f ? (long long)ceilf(reach) + 3 : (1ll << 40);
                const int n[3] = {a.nx, a.ny, a.nz};
                for (int r = 0; r < 3; ++r) {
                    const long long lo = E - s_omin[r], hi = (long long)(n[r] - 2) - E - s_omax[r];
                    s_lo[r] = (int)(lo > INT_MAX ? INT_MAX : (lo < INT_MIN ? INT_MIN : lo));
                    s_hi[r] = (int)(hi < INT_MIN ? INT_MIN : (hi > INT_MAX ? INT_MAX : hi));
                }
            }
            __syncthreads();
            const int lo[3] = {s_lo[0], s_lo[1], s_lo[2]}, hi[3] = {s_hi[0], s_hi[1], s_hi[2]};
            // reference products, interior flags and pairs (point p, point p + 2)
            PointPair P2[PPT / 2];
            int Yi[PPT][3];
            bool in_all = true;
#pragma unroll
            for (int h = 0; h < PPT / 2; ++h) {
                int* Ya = Yi[h];
                int* Yb = Yi[h + 2];
                float Fa[3], Fb[3];
                ref_apply(sRef, px[h], py[h], pz[h], Ya, Fa);
                ref_apply(sRef, px[h + 2], py[h + 2], pz[h + 2], Yb, Fb);
                const bool ia = point_interior(Ya, Fa, lo, hi), ib = point_interior(Yb, Fb, lo, hi);
                in_all = in_all && ia && ib;
                P2[h].x = make_float2(px[h], px[h + 2]);
                P2[h].y = make_float2(py[h], py[h + 2]);
                P2[h].z = make_float2(pz[h], pz[h + 2]);
                P2[h].yf0 = make_float2(Fa[0], Fb[0]);
                P2[h].yf1 = make_float2(Fa[1], Fb[1]);
                P2[h].yf2 = make_float2(Fa[2], Fb[2]);
                P2[h].yla = (ia && ib) ? linear_cell(Ya, nx, nxy) : INT_MIN;
                P2[h].ylb = linear_cell(Yb, nx, nxy);
            }
            if (!s_mode) {
                if (__all_sync(0xffffffffu, in_all)) {
                    for (int kk = 0; kk < kc; ++kk) {
                        XformD X;
                        load_xformd(sPD[kk], X);
                        float s = 0.0f;
                        int c = 0;
#pragma unroll
                        for (int h = 0; h < PPT / 2; ++h) {
                            Cell ca, cb;
                            locate2<false>(X, nx, nxy, mx, my, mz, P2[h], nullptr, nullptr, ca, cb);
                            gather<VARIANT, TS, true>(a, nx, nxy, ca, s, c);
                            gather<VARIANT, TS, true>(a, nx, nxy, cb, s, c);
                        }
                        c = __reduce_add_sync(0xffffffffu, c);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                        if (lane == 0) {
                            accS[warp][kk] += s;
                            accC[warp][kk] += c;
                        }
                    }
                } else {
                    // some point of the warp may leave the grid: per-sample
                    // range tests
                    for (int kk = 0; kk < kc; ++kk) {
                        XformD X;
                        load_xformd(sPD[kk], X);
                        float s = 0.0f;
                        int c = 0;
#pragma unroll
                        for (int h = 0; h < PPT / 2; ++h) {
                            Cell ca, cb;
                            locate2<true>(X, nx, nxy, mx, my, mz, P2[h], Yi[h], Yi[h + 2], ca, cb);
                            gather<VARIANT, TS, true>(a, nx, nxy, ca, s, c);
                            gather<VARIANT, TS, true>(a, nx, nxy, cb, s, c);
                        }
                        c = __reduce_add_sync(0xffffffffu, c);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                        if (lane == 0) {
                            accS[warp][kk] += s;
                            accC[warp][kk] += c;
                        }
                    }
                }
            } else {
                // the warp's 128 points as 64 pairs: pair h * 32 + lane holds
                // this lane's points h and h + 2
#pragma unroll
                for (int h = 0; h < PPT / 2; ++h) {
                    const int j = h * 32 + lane;
                    sPair[warp][j][0] = make_float4(P2[h].x.x, P2[h].x.y, P2[h].y.x, P2[h].y.y);
                    sPair[warp][j][1] = make_float4(P2[h].z.x, P2[h].z.y, P2[h].yf0.x, P2[h].yf0.y);
                    sPair[warp][j][2] = make_float4(P2[h].yf1.x, P2[h].yf1.y, P2[h].yf2.x, P2[h].yf2.y);
                    sPyl[warp][j] = make_int2(P2[h].yla, P2[h].ylb);
                }
                __syncwarp();
                const int kl = lane < kc ? lane : 0;
                XformD X;
                load_xformd(sPD[kl], X);
                float s = 0.0f;
                int c = 0;
                // 16-/8-bit grids: lanes on particles read the float records
                // of a full view (no conversions; for 16-bit storage the
                // same samples bit for bit), else the narrow records; the
                // loops are instantiated once per source so that the choice
                // costs the inner loop nothing
                auto pair_loops = [&](auto float_cells) {
                    constexpr bool FC = decltype(float_cells)::value;
                    if (__all_sync(0xffffffffu, in_all)) {
                        // every pair of the warp is interior: no range tests
#pragma unroll 4
                        for (int j = 0; j < PPT * 16; ++j) {
                            const float4 q0 = sPair[warp][j][0], q1 = sPair[warp][j][1], q2 = sPair[warp][j][2];
                            const int2 yl = sPyl[warp][j];
                            PointPair pp;
                            pp.x = make_float2(q0.x, q0.y);
                            pp.y = make_float2(q0.z, q0.w);
                            pp.z = make_float2(q1.x, q1.y);
                            pp.yf0 = make_float2(q1.z, q1.w);
                            pp.yf1 = make_float2(q2.x, q2.y);
                            pp.yf2 = make_float2(q2.z, q2.w);
                            pp.yla = yl.x;
                            pp.ylb = yl.y;
                            Cell ca, cb;
                            locate2<false>(X, nx, nxy, mx, my, mz, pp, nullptr, nullptr, ca, cb);
                            gather<VARIANT, TS, true, FC>(a, nx, nxy, ca, s, c);
                            gather<VARIANT, TS, true, FC>(a, nx, nxy, cb, s, c);
                        }
                    } else {
#pragma unroll 2
                        for (int j = 0; j < PPT * 16; ++j) {
                            const float4 q0 = sPair[warp][j][0], q1 = sPair[warp][j][1], q2 = sPair[warp][j][2];
                            const int2 yl = sPyl[warp][j];
                            PointPair pp;
                            pp.x = make_float2(q0.x, q0.y);
                            pp.y = make_float2(q0.z, q0.w);
                            pp.z = make_float2(q1.x, q1.y);
                            pp.yf0 = make_float2(q1.z, q1.w);
                            pp.yf1 = make_float2(q2.x, q2.y);
                            pp.yf2 = make_float2(q2.z, q2.w);
                            pp.yla = yl.x;
                            pp.ylb = yl.y;
                            Cell ca, cb;
                            if (yl.x != INT_MIN) {  // the same for every lane
                                locate2<false>(X, nx, nxy, mx, my, mz, pp, nullptr, nullptr, ca, cb);
                            } else {
                                // a pair near the grid's edge (rare): the
                                // reference cells again, from the points
                                int Ya[3], Yb[3];
                                float Fa[3], Fb[3];
                                ref_apply(sRef, pp.x.x, pp.y.x, pp.z.x, Ya, Fa);
                                ref_apply(sRef, pp.x.y, pp.y.y, pp.z.y, Yb, Fb);
                                locate2<true>(X, nx, nxy, mx, my, mz, pp, Ya, Yb, ca, cb);
                            }
                            gather<VARIANT, TS, true, FC>(a, nx, nxy, ca, s, c);
                            gather<VARIANT, TS, true, FC>(a, nx, nxy, cb, s, c);
                        }
                    }
                };
                if constexpr (!std::is_same<TS, float>::value) {
                    if (a.cells32 != nullptr)
                        pair_loops(std::true_type{});
                    else
                        pair_loops(std::false_type{});
                } else {
                    pair_loops(std::false_type{});
                }
                __syncwarp();
                if (lane < kc) {
                    accS[warp][lane] += s;
                    accC[warp][lane] += c;
                }
            }
        }
    }
    __syncthreads();
    if (tid < kc) {
        float S = 0.0f;
        int C = 0;
        for (int w = 0; w < FIT_WARPS; ++w) {
            S += accS[w][tid];
            C += accC[w][tid];
        }
        const size_t slot = (size_t)by * a.K + k_begin + tid;
        a.part_S[slot] = S;
        a.part_C[slot] = C;
    }
    __threadfence();
    __syncthreads();
    const bool two_level = SOLO && SRC == SRC_SEARCH && a.chunk_counter != nullptr;
    if (two_level) {
        // the last of the chunk's point tiles reduces the chunk's particles
        // over the tiles (in parallel with other chunks' sampling) ...
        if (tid == 0) {
            const unsigned int ticket = atomicAdd(a.chunk_counter + bx, 1u);
            s_last = ticket == (unsigned)a.n_ptiles - 1;
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        if (tid < kc) {
            float S;
            int C;
            sum_tiles(a.part_S, a.part_C, a.K, a.n_ptiles, k_begin + tid, S, C);
            a.chunk_E[k_begin + tid] = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
            a.chunk_C[k_begin + tid] = C;
        }
        if (tid == 0) a.chunk_counter[bx] = 0u;
        __threadfence();
        __syncthreads();
        // ... and the last chunk to finish runs the selection below
        if (tid == 0) {
            const unsigned int ticket = atomicAdd(a.counter, 1u);
            s_last = ticket == (unsigned)((a.K + KC - 1) / KC) - 1;
        }
    } else {
        if (tid == 0) {
            const unsigned int ticket = atomicAdd(a.counter, 1u);
            s_last = ticket == n_blocks - 1;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ------------------------------------------------------------------
    // Last CTA: reduce partials over point tiles (fixed order) and finish.
    // ------------------------------------------------------------------
    if (SRC == SRC_POSES) {
        for (int k = tid; k < a.K; k += FIT_THREADS) {
            float S;
            int C;
            sum_tiles(a.part_S, a.part_C, a.K, a.n_ptiles, k, S, C);
            a.out_E[k] = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
            a.out_C[k] = C;
        }
    } else if (SRC == SRC_EVAL) {
        // one pose over up to a few hundred tiles: every thread sums tiles
        // tid, tid + 256, ... and the block combines the sums in a fixed order
        __shared__ float s_eS[FIT_WARPS];
        __shared__ int s_eC[FIT_WARPS];
        float S = 0.0f;
        int C = 0;
        for (int y = tid; y < a.n_ptiles; y += FIT_THREADS) {
            S += __ldcg(a.part_S + y);
            C += __ldcg(a.part_C + y);
        }
        for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        C = __reduce_add_sync(0xffffffffu, C);
        if (lane == 0) {
            s_eS[warp] = S;
            s_eC[warp] = C;
        }
        __syncthreads();
        if (tid == 0) {
            if (!skip) {
                S = 0.0f;
                C = 0;
                for (int w = 0; w < FIT_WARPS; ++w) {
                    S += s_eS[w];
                    C += s_eC[w];
                }
                const float E = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
                SearchState* st = a.st;
                const double e = isfinite(E) ? (double)E : 1.0;
                const double f = a.beta + (1.0 - a.beta) * e;
                st->s[0] *= f;
                st->s[1] *= f;
                st->pending_s = 0;
                a.stats->E_new[a.iter] = E;
            }
        }
    } else {  // SRC_SEARCH
        __shared__ float s_E0;
        __shared__ int s_C0;
        __shared__ float se[FIT_WARPS];
        __shared__ int sk[FIT_WARPS];
        __shared__ double sd[FIT_WARPS][6];
        __shared__ int sn[FIT_WARPS];
        SearchState* st = a.st;
        if (tid == 0) {
            if (two_level) {
                s_E0 = __ldcg(a.chunk_E);
                s_C0 = __ldcg(a.chunk_C);
            } else {
                float S;
                int C;
                sum_tiles(a.part_S, a.part_C, a.K, a.n_ptiles, 0, S, C);
                s_E0 = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
                s_C0 = C;
            }
        }
        __syncthreads();
        const float E0 = s_E0;
        float be = INFINITY;
        int bk = 0x7fffffff;
        int nadv = 0;
        double sum[6] = {0, 0, 0, 0, 0, 0};
        for (int k = tid; k < a.K; k += FIT_THREADS) {
            float E;
            if (two_level) {
                E = __ldcg(a.chunk_E + k);
            } else {
                float S;
                int C;
                sum_tiles(a.part_S, a.part_C, a.K, a.n_ptiles, k, S, C);
                E = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
            }
            if (E < be) {
                be = E;
                bk = k;
            }
            if (E < E0) {
                ++nadv;
                const float* u = a.templ + 6 * (size_t)k;
                for (int q = 0; q < 6; ++q) sum[q] += (double)u[q];
            }
        }
        if (bk == 0x7fffffff) bk = 0;  // all +inf on this thread: any index, ties resolve to 0 below
        argmin_pair(be, bk, se, sk);
        // deterministic block sums of nadv and the template sums
        for (int o = 16; o > 0; o >>= 1) {
            nadv += __shfl_xor_sync(0xffffffffu, nadv, o);
            for (int q = 0; q < 6; ++q) sum[q] += __shfl_xor_sync(0xffffffffu, sum[q], o);
        }
        if (lane == 0) {
            sn[warp] = nadv;
            for (int q = 0; q < 6; ++q) sd[warp][q] = sum[q];
        }
        __syncthreads();
        if (tid == 0 && !skip) {
            int n_adv = 0;
            double mu[6] = {0, 0, 0, 0, 0, 0};
            for (int w = 0; w < FIT_WARPS; ++w) {
                n_adv += sn[w];
                for (int q = 0; q < 6; ++q) mu[q] += sd[w][q];
            }
            pf_track_stats* stt = a.stats;
            const int it = a.iter;
            const long long nev = Ne;
            const double s_deg = st->s[0], s_cm = st->s[1];
            stt->n_points = N;
            stt->E0[it] = E0;
            stt->E_best[it] = be;
            stt->best[it] = bk;
            stt->n_adv[it] = n_adv;
            stt->n_valid0[it] = s_C0;
            stt->n_eval[it] = (int)nev;
            stt->k_used[it] = a.K;
            stt->s[it][0] = s_deg;
            stt->s[it][1] = s_cm;
            stt->n_iters = it + 1;
            const bool lost = it == 0 && (!isfinite(E0) || (double)s_C0 < (double)a.min_valid_frac * (double)nev);
            if (lost) {
                st->lost = 1;
                stt->E_new[it] = INFINITY;
                for (int q = 0; q < 12; ++q) stt->pose[it][q] = st->P0[q];
            } else {
                const double wr = s_deg * kPi / 180.0, wt = s_cm / 100.0;
                double dw[3], dt[3];
                bool moved = true;
                if (a.update_mode == 1) {
                    const float* u = a.templ + 6 * (size_t)bk;
                    for (int q = 0; q < 3; ++q) {
                        dw[q] = wr * (double)u[q];
                        dt[q] = wt * (double)u[3 + q];
                    }
                } else if (n_adv > 0) {
                    for (int q = 0; q < 3; ++q) {
                        dw[q] = wr * (mu[q] / n_adv);
                        dt[q] = wt * (mu[3 + q] / n_adv);
                    }
                } else {
                    moved = false;
                }
                if (moved) {
                    double dR[9], Pn[12];
                    so3_exp_d(dw, dR);
                    compose_d(dR, dt, st->P, a.compose_mode, Pn);
                    for (int q = 0; q < 12; ++q) st->P[q] = Pn[q];
                }
                for (int q = 0; q < 12; ++q) stt->pose[it][q] = st->P[q];
                if (a.update_mode == 1 || !moved) {
                    const float En = a.update_mode == 1 ? be : E0;
                    const double e = isfinite(En) ? (double)En : 1.0;
                    const double f = a.beta + (1.0 - a.beta) * e;
                    st->s[0] *= f;
                    st->s[1] *= f;
                    stt->E_new[it] = En;
                    st->pending_s = 0;
                } else {
                    st->pending_s = 1;
                }
            }
        }
    }
    if (tid == 0) *a.counter = 0u;
}

template <int SRC, int VARIANT, typename TS>
__global__ void __launch_bounds__(FIT_THREADS, PF_FIT_MIN_BLOCKS) fitness_kernel(FitArgs a)
{
    fitness_body<SRC, VARIANT, TS, true>(a, blockIdx.x, blockIdx.y, gridDim.x * gridDim.y);
}

// One launch over the CTAs of several independent problems (the sequences
// of a batch): problem i owns CTAs [first[i], first[i + 1]), chunk-fastest,
// with its own arguments, partials, ticket counter and epilogue, so each
// problem's results are those of its own launch.
template <int SRC, int VARIANT, typename TS>
__global__ void __launch_bounds__(FIT_THREADS, PF_FIT_MIN_BLOCKS)
    fitness_kernel_batch(const FitArgs* __restrict__ args, const int* __restrict__ first, int n)
{
    __shared__ FitArgs sa;
    __shared__ int s_id;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;  // the last problem with first[i] <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= (int)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_id = lo;
    }
    __syncthreads();
    const int id = s_id;
    static_assert(sizeof(FitArgs) % 4 == 0, "FitArgs is copied as words");
    const int* src = reinterpret_cast<const int*>(args + id);
    int* dst = reinterpret_cast<int*>(&sa);
    for (int q = threadIdx.x; q < (int)(sizeof(FitArgs) / 4); q += FIT_THREADS) dst[q] = __ldg(src + q);
    __syncthreads();
    const int local = (int)blockIdx.x - __ldg(first + id);
    const int chunks = (sa.K + KC - 1) / KC;
    fitness_body<SRC, VARIANT, TS, false>(sa, local % chunks, local / chunks, (unsigned)(chunks * sa.n_ptiles));
}

__global__ void track_begin_kernel(SearchState* st, const double* P0, double s_deg, double s_cm,
                                   pf_track_stats* stats)
{
    if (threadIdx.x == 0) {
        for (int q = 0; q < 12; ++q) {
            st->P[q] = P0[q];
            st->P0[q] = P0[q];
        }
        st->s[0] = s_deg;
        st->s[1] = s_cm;
        st->lost = 0;
        st->pending_s = 0;
        stats->n_iters = 0;
        stats->status = PF_OK;
        stats->n_points = 0;
    }
}

__global__ void track_end_kernel(const SearchState* st, const int* n_points, double* out_pose,
                                 pf_track_stats* stats)
{
    if (threadIdx.x == 0) {
        const double* P = st->lost ? st->P0 : st->P;
        for (int q = 0; q < 12; ++q) out_pose[q] = P[q];
        out_pose[12] = 0.0;
        out_pose[13] = 0.0;
        out_pose[14] = 0.0;
        out_pose[15] = 1.0;
        stats->status = st->lost ? PF_ERR_TRACK_LOST : PF_OK;
        stats->n_points = *n_points;
    }
}

int device_sms(int dev)
{
    static int cached_dev = -1, cached_n = 0;
    if (dev == cached_dev) return cached_n;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cached_dev = dev;
    cached_n = n;
    return n;
}

// Point tiles of a launch (the rule and its bound: ptiles.h), for this
// device's resident CTA slots.
int choose_ptiles(int dev, int chunks, long long ne_max)
{
    return pf::choose_ptiles_for((long long)device_sms(dev) * PF_FIT_MIN_BLOCKS, SUBTILE, chunks, ne_max);
}

int ptiles_bound(int dev, int chunks, long long ne_max)
{
    return pf::ptiles_bound_for((long long)device_sms(dev) * PF_FIT_MIN_BLOCKS, SUBTILE, chunks, ne_max);
}

// variant = layout + 4 * mapping (see pf_set_fitness_variant).  Measured on
// the 640x480 / 512^3 workload, particles on lanes win below a spread of
// about 0.5 degree and 0.5 cm with the cell view (~5 voxels by the bound
// used here) and below about 1 degree and 1 cm on the node array (~12).
constexpr float kParticleLanesBelowCells = 5.0f;
constexpr float kParticleLanesBelowNodes = 12.0f;

template <int SRC, typename TS>
void launch_fitness_t(const FitArgs& a, int layout, dim3 grid, cudaStream_t s)
{
    if (layout == 2)
        fitness_kernel<SRC, 0, TS><<<grid, FIT_THREADS, 0, s>>>(a);
    else
        fitness_kernel<SRC, 2, TS><<<grid, FIT_THREADS, 0, s>>>(a);
}

// Layout the fitness of this volume runs with (see pf_set_fitness_variant).
int resolve_fitness_layout(const pf_volume* v)
{
    const int layout = v->fitness_variant & 3;
    return layout == 0 ? (v->cells ? 3 : 2) : layout;
}

template <int SRC>
void launch_fitness(FitArgs a, int variant, const pf_volume* v, int chunks, cudaStream_t s)
{
    const int mapping = (variant >> 2) & 3;
    int layout = variant & 3;
    if (layout == 0) layout = v->cells ? 3 : 2;
    const float auto_threshold = layout == 3 ? kParticleLanesBelowCells : kParticleLanesBelowNodes;
    a.pm_threshold = mapping == 1 ? -1.0f : mapping == 2 ? INFINITY : auto_threshold;
    dim3 grid(chunks, a.n_ptiles);
    const pf_dtype dt = pf_fitness_dtype(v, layout);  // the cell view's records, or the node array's values
    if (layout == 1)  // the plain baseline: float tsdf and weights
        fitness_kernel<SRC, 1, float><<<grid, FIT_THREADS, 0, s>>>(a);
    else if (dt == PF_F16)
        launch_fitness_t<SRC, __half>(a, layout, grid, s);
    else if (dt == PF_BF16)
        launch_fitness_t<SRC, __nv_bfloat16>(a, layout, grid, s);
    else if (dt == PF_FP8E4M3)
        launch_fitness_t<SRC, __nv_fp8_e4m3>(a, layout, grid, s);
    else
        launch_fitness_t<SRC, float>(a, layout, grid, s);
    pf::count_launch();
}

void fill_volume_args(FitArgs& a, const pf_volume* v)
{
    a.tsdf = v->tsdf;
    a.weight = v->weight;
    a.cells = v->cells;
    a.cells32 = v->cells32;
    a.nx = v->desc.nx;
    a.ny = v->desc.ny;
    a.nz = v->desc.nz;
    a.vs = v->desc.voxel_size;
    for (int q = 0; q < 3; ++q) a.org[q] = v->desc.origin[q];
}

pf_status grow_partials(pf_volume* v, size_t need)
{
    pf_workspace& w = v->ws;
    if ((size_t)w.part_cap >= need && w.counter) return PF_OK;
    PF_CUDA(cudaDeviceSynchronize());
    if (!w.counter) {
        PF_CUDA(pf::dev_malloc(&w.counter, sizeof(unsigned int)));
        PF_CUDA(cudaMemset(w.counter, 0, sizeof(unsigned int)));
    }
    if ((size_t)w.part_cap < need) {
        cudaFree(w.part_S);
        cudaFree(w.part_C);
        w.part_S = nullptr;
        w.part_C = nullptr;
        w.part_cap = 0;
        PF_CUDA(pf::dev_malloc(&w.part_S, need * sizeof(float)));
        PF_CUDA(pf::dev_malloc(&w.part_C, need * sizeof(int)));
        w.part_cap = (int)need;
    }
    return PF_OK;
}

pf_status check_params(const pf_track_params* p)
{
    if (!p || !p->templates_dev) return PF_ERR_INVALID_ARG;
    if (p->n_iters < 1 || p->n_iters > PF_MAX_ITERS) return PF_ERR_INVALID_ARG;
    if (p->k_max < 1 || p->k_max > 65536) return PF_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i) {
        if (p->k_sched[i] < 1 || p->k_sched[i] > p->k_max) return PF_ERR_INVALID_ARG;
        if (p->decim_sched[i] < 1) return PF_ERR_INVALID_ARG;
    }
    if (!(p->init_rot_deg >= 0.0) || !(p->init_trans_cm >= 0.0) || !std::isfinite(p->init_rot_deg) ||
        !std::isfinite(p->init_trans_cm))
        return PF_ERR_INVALID_ARG;
    if (!(p->beta >= 0.0 && p->beta <= 1.0)) return PF_ERR_INVALID_ARG;
    if (p->update_mode < 0 || p->update_mode > 1 || p->compose_mode < 0 || p->compose_mode > 1)
        return PF_ERR_INVALID_ARG;
    if (!(p->min_valid_frac >= 0.0f && p->min_valid_frac <= 1.0f)) return PF_ERR_INVALID_ARG;
    return PF_OK;
}

}  // namespace

namespace pf {

pf_status workspace_reserve(pf_volume* v, int max_pixels, int k_max)
{
    if (!v || max_pixels < 1 || k_max < 1) return PF_ERR_INVALID_ARG;
    pf_workspace& w = v->ws;
    const long long ne_max = max_pixels;
    // partial slots: the largest tiles x particles over every particle count
    // up to k_max and every point count up to max_pixels
    size_t need = 0;
    for (int chunks = 1; chunks <= (k_max + KC - 1) / KC; ++chunks) {
        const size_t K = std::min((size_t)chunks * KC, (size_t)k_max);
        need = std::max(need, (size_t)ptiles_bound(v->device, chunks, ne_max) * K);
    }
    pf_status st = grow_partials(v, need);
    if (st != PF_OK) return st;
    const int chunks_needed = (k_max + KC - 1) / KC;
    if (w.chunk_cap < chunks_needed) {
        PF_CUDA(cudaDeviceSynchronize());
        cudaFree(w.chunks);
        w.chunks = nullptr;
        w.chunk_cap = 0;
        cudaFree(w.chunk_counter);
        cudaFree(w.chunk_E);
        cudaFree(w.chunk_C);
        w.chunk_counter = nullptr;
        w.chunk_E = nullptr;
        w.chunk_C = nullptr;
        PF_CUDA(pf::dev_malloc(reinterpret_cast<ChunkData**>(&w.chunks), sizeof(ChunkData) * (size_t)chunks_needed));
        PF_CUDA(pf::dev_malloc(&w.chunk_counter, sizeof(unsigned int) * (size_t)chunks_needed));
        PF_CUDA(cudaMemset(w.chunk_counter, 0, sizeof(unsigned int) * (size_t)chunks_needed));
        PF_CUDA(pf::dev_malloc(&w.chunk_E, sizeof(float) * KC * (size_t)chunks_needed));
        PF_CUDA(pf::dev_malloc(&w.chunk_C, sizeof(int) * KC * (size_t)chunks_needed));
        w.chunk_cap = chunks_needed;
    }
    if (w.pix_cap < max_pixels) {
        PF_CUDA(cudaDeviceSynchronize());
        cudaFree(w.points);
        cudaFree(w.block_counts);
        cudaFree(w.point_tile);
        cudaFree(w.kept);
        cudaFree(w.kept_count);
        cudaFree(w.order_scratch);
        w.points = nullptr;
        w.block_counts = nullptr;
        w.point_tile = nullptr;
        w.kept = nullptr;
        w.kept_count = nullptr;
        w.order_scratch = nullptr;
        w.order_cap = 0;
        w.pix_cap = 0;
        PF_CUDA(pf::dev_malloc(&w.point_tile, sizeof(int) * (size_t)max_pixels));
        PF_CUDA(pf::dev_malloc(&w.kept, 2 * sizeof(float4) * (size_t)max_pixels));
        PF_CUDA(pf::dev_malloc(&w.kept_count, 4 * sizeof(int)));
        const size_t slots = kept_slots_bound((size_t)max_pixels);
        PF_CUDA(pf::dev_malloc(&w.order_scratch, 3 * sizeof(int) * slots));
        w.order_cap = (int)slots;
        PF_CUDA(pf::dev_malloc(&w.points, sizeof(float4) * (size_t)max_pixels));
        // one count per back-projection block: an image of max_pixels pixels has
        // at most max_pixels tiles (thin images leave tiles partly empty)
        PF_CUDA(pf::dev_malloc(&w.block_counts, sizeof(int) * ((size_t)max_pixels / BP_CHUNK_TILES + 2)));
        w.pix_cap = max_pixels;
    }
    if (!w.state) {
        PF_CUDA(pf::dev_malloc(&w.state, sizeof(SearchState)));
        PF_CUDA(pf::dev_malloc(&w.n_points, sizeof(int)));
        PF_CUDA(pf::dev_malloc(&w.pose_in, 16 * sizeof(double)));
        PF_CUDA(pf::dev_malloc(&w.pose_out, 16 * sizeof(double)));
        PF_CUDA(pf::dev_malloc(&w.stats, sizeof(pf_track_stats)));
        PF_CUDA(cudaMemset(w.stats, 0, sizeof(pf_track_stats)));
    }
    w.k_cap = std::max(w.k_cap, k_max);
    return PF_OK;
}

}  // namespace pf

extern "C" {

pf_status pf_backproject(const float* depth_dev, const pf_intrinsics* intr, float* points_dev, int capacity,
                         int* n_dev, void* stream)
{
    if (!depth_dev || !points_dev || !n_dev) return PF_ERR_INVALID_ARG;
    pf_status st = pf::check_intrinsics(intr);
    if (st != PF_OK) return st;
    const long long npix = (long long)intr->width * intr->height;
    if (capacity < npix) return PF_ERR_INVALID_ARG;
    int* counts = nullptr;
    const int blocks = bp_blocks(intr->width, intr->height);
    PF_CUDA(pf::dev_malloc_async(&counts, sizeof(int) * blocks, (cudaStream_t)stream));
    st = enqueue_backproject(depth_dev, intr, reinterpret_cast<float4*>(points_dev), counts, n_dev,
                             (cudaStream_t)stream);
    cudaFreeAsync(counts, (cudaStream_t)stream);
    return st;
}

static pf_status pf_fitness_impl(const pf_volume* cv, const float* points_dev, int n, const float* poses_dev, int k,
                                 float* fitness_dev, int* count_dev, void* stream)
{
    pf_volume* v = const_cast<pf_volume*>(cv);
    if (!v || !poses_dev || !fitness_dev || !count_dev) return PF_ERR_INVALID_ARG;
    if (n < 0 || k < 1 || k > 65536 || (n > 0 && !points_dev)) return PF_ERR_INVALID_ARG;
    const int chunks = (k + KC - 1) / KC;
    const int tiles = choose_ptiles(v->device, chunks, n);
    pf_status st = grow_partials(v, (size_t)tiles * k);
    if (st != PF_OK) return st;
    FitArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = reinterpret_cast<const float4*>(points_dev);
    a.n_dev = nullptr;
    a.n_host = n;
    a.stride = 1;
    a.K = k;
    a.poses = poses_dev;
    fill_volume_args(a, v);
    a.part_S = v->ws.part_S;
    a.part_C = v->ws.part_C;
    a.counter = v->ws.counter;
    a.n_ptiles = tiles;
    a.out_E = fitness_dev;
    a.out_C = count_dev;
    cudaStream_t s = (cudaStream_t)stream;
    pf::timing_begin(pf::KC_FITNESS, s);
    launch_fitness<SRC_POSES>(a, v->fitness_variant, v, chunks, s);
    pf::timing_end(pf::KC_FITNESS, s);
    PF_LAUNCHED();
    return PF_OK;
}

static pf_status pf_track_reserve_impl(pf_volume* v, int max_pixels, int k_max)
{
    return pf::workspace_reserve(v, max_pixels, k_max);
}

static pf_status pf_track_frame_async_impl(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr,
                                           const pf_track_params* p, const double* init_pose_dev,
                                           double* out_pose_dev, pf_track_stats* stats_dev, void* stream)
{
    if (!v || !depth_dev || !init_pose_dev || !out_pose_dev) return PF_ERR_INVALID_ARG;
    pf_status st = pf::check_intrinsics(intr);
    if (st != PF_OK) return st;
    st = check_params(p);
    if (st != PF_OK) return st;
    const int npix = intr->width * intr->height;
    pf_workspace& w = v->ws;
    if (w.pix_cap < npix || w.k_cap < p->k_max || !w.state) {
        st = pf::workspace_reserve(v, std::max(npix, w.pix_cap), std::max(p->k_max, w.k_cap));
        if (st != PF_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    pf_track_stats* stats = stats_dev ? stats_dev : w.stats;
    SearchState* state = reinterpret_cast<SearchState*>(w.state);

    track_begin_kernel<<<1, 32, 0, s>>>(state, init_pose_dev, p->init_rot_deg, p->init_trans_cm, stats);
    pf::count_launch();
    st = enqueue_backproject(depth_dev, intr, w.points, w.block_counts, w.n_points, s, w.point_tile);
    if (st != PF_OK) return st;
    // the decimated point sets of the schedule, each in a locality order
    int kept_stride[3] = {0, 0, 0};
    const float4* kept_pts[3] = {nullptr, nullptr, nullptr};
    int n_kept = 0;
    size_t kept_off = 0;
    for (int i = 0; i < 3; ++i) {
        const int n = p->decim_sched[i];
        bool seen = false;
        for (int d = 0; d < n_kept; ++d) seen = seen || kept_stride[d] == n;
        if (n <= 1 || n > kMaxOrderedStride || seen) continue;
        const KeptOrder o = kept_order(n, intr->width, intr->height);
        if (o.n_slots > w.order_cap) continue;  // (cannot happen within the bound; strided reading then)
        int* cnt = w.order_scratch;
        int* first = cnt + w.order_cap;
        int* offset = first + w.order_cap;
        const int ne_max = (npix + n - 1) / n;
        const int grid = std::max(1, std::min(1024, (ne_max + 255) / 256));
        pf::timing_begin(pf::KC_BACKPROJECT, s);
        kept_clear_kernel<<<std::max(1, std::min(1024, (o.n_slots + 255) / 256)), 256, 0, s>>>(cnt, first, o.n_slots);
        kept_count_kernel<<<grid, 256, 0, s>>>(o, w.n_points, w.point_tile, cnt, first);
        kept_scan_kernel<<<1, 256, 0, s>>>(cnt, offset, o.n_slots);
        kept_write_kernel<<<grid, 256, 0, s>>>(o, w.n_points, w.points, w.point_tile, first, offset,
                                               w.kept + kept_off, w.kept_count + n_kept);
        pf::count_launch(4);
        pf::timing_end(pf::KC_BACKPROJECT, s);
        PF_LAUNCHED();
        kept_stride[n_kept] = n;
        kept_pts[n_kept] = w.kept + kept_off;
        kept_off += (size_t)ne_max;
        ++n_kept;
    }

    FitArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = w.points;
    a.n_dev = w.n_points;
    a.templ = p->templates_dev;
    a.st = state;
    a.compose_mode = p->compose_mode;
    a.update_mode = p->update_mode;
    a.beta = p->beta;
    a.min_valid_frac = p->min_valid_frac;
    fill_volume_args(a, v);
    a.part_S = w.part_S;
    a.part_C = w.part_C;
    a.counter = w.counter;
    a.stats = stats;
    for (int it = 0; it < p->n_iters; ++it) {
        const int K = p->k_sched[it % 3];
        const int stride = p->decim_sched[it % 3];
        const long long ne_max = ((long long)npix + stride - 1) / stride;
        const int chunks = (K + KC - 1) / KC;
        a.K = K;
        a.pts = w.points;
        a.n_dev = w.n_points;
        a.stride = stride;
        for (int d = 0; d < n_kept; ++d)
            if (kept_stride[d] == stride) {  // the kept points, already in their locality order
                a.pts = kept_pts[d];
                a.n_dev = w.kept_count + d;
                a.stride = 1;
            }
        a.iter = it;
        a.n_ptiles = choose_ptiles(v->device, chunks, ne_max);
        if ((size_t)a.n_ptiles * K > (size_t)w.part_cap || chunks > w.chunk_cap) return PF_ERR_INVALID_ARG;
        // the iteration's particles, built once (the plain baseline layout
        // builds its own in every CTA, as it always did)
        const bool prebuild = resolve_fitness_layout(v) != 1;
        a.chunks = prebuild ? w.chunks : nullptr;
        a.chunk_counter = w.chunk_counter;
        a.chunk_E = w.chunk_E;
        a.chunk_C = w.chunk_C;
        pf::timing_begin(pf::KC_FITNESS, s);
        if (prebuild) {
            chunk_build_kernel<SRC_SEARCH><<<chunks, 32, 0, s>>>(a, static_cast<ChunkData*>(w.chunks));
            pf::count_launch();
        }
        launch_fitness<SRC_SEARCH>(a, v->fitness_variant, v, chunks, s);
        pf::timing_end(pf::KC_FITNESS, s);
        if (p->update_mode == 0) {
            FitArgs e = a;
            e.chunks = nullptr;  // one particle, built in its CTAs, reduced by the launch's last CTA
            e.chunk_counter = nullptr;
            e.chunk_E = nullptr;
            e.chunk_C = nullptr;
            e.K = 1;
            e.n_ptiles = choose_ptiles(v->device, 1, ne_max);
            pf::timing_begin(pf::KC_FITNESS1, s);
            launch_fitness<SRC_EVAL>(e, v->fitness_variant, v, 1, s);
            pf::timing_end(pf::KC_FITNESS1, s);
        }
    }
    track_end_kernel<<<1, 32, 0, s>>>(state, w.n_points, out_pose_dev, stats);
    pf::count_launch();
    PF_LAUNCHED();
    return PF_OK;
}

static pf_status pf_track_frame_impl(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr,
                                     const pf_track_params* p, const double init_pose[16], double out_pose[16],
                                     pf_track_stats* stats_host, void* stream)
{
    if (!v || !init_pose || !out_pose) return PF_ERR_INVALID_ARG;
    for (int q = 0; q < 12; ++q)
        if (!std::isfinite(init_pose[q])) return PF_ERR_INVALID_ARG;
    pf_status st = pf::check_intrinsics(intr);
    if (st != PF_OK) return st;
    st = check_params(p);
    if (st != PF_OK) return st;
    const int npix = intr->width * intr->height;
    pf_workspace& w = v->ws;
    if (w.pix_cap < npix || w.k_cap < p->k_max || !w.state) {
        st = pf::workspace_reserve(v, std::max(npix, w.pix_cap), std::max(p->k_max, w.k_cap));
        if (st != PF_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    PF_CUDA(cudaMemcpyAsync(w.pose_in, init_pose, 16 * sizeof(double), cudaMemcpyHostToDevice, s));
    st = pf_track_frame_async(v, depth_dev, intr, p, w.pose_in, w.pose_out, w.stats, stream);
    if (st != PF_OK) return st;
    pf_track_stats hs;
    PF_CUDA(cudaMemcpyAsync(out_pose, w.pose_out, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaMemcpyAsync(&hs, w.stats, sizeof(pf_track_stats), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    if (stats_host) *stats_host = hs;
    return hs.status == PF_ERR_TRACK_LOST ? PF_ERR_TRACK_LOST : PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many independent sequences stepped together
// ---------------------------------------------------------------------------
namespace pf {
bool timing_swap(bool enabled);  // api.cu
}

struct pf_batch {
    int n = 0;
    std::vector<pf_volume*> vols;
    std::vector<pf_intrinsics> intrs;
    std::vector<pf_track_params> params;
    int max_iters = 0;
    int layout = 3;
    pf_dtype dtype = PF_F32;
    int device = 0;
    // device buffers: depth images (one allocation), per sequence four poses
    // (relative input, current pose, initial pose of the search, spare) and
    // the search record
    float* depth = nullptr;
    std::vector<size_t> depth_off;
    double* poses = nullptr;
    pf_track_stats* stats = nullptr;
    // launch tables, per iteration: arguments of every participating
    // sequence and the first CTA of each (search, then single-pose
    // evaluation for the mean update)
    FitArgs* d_args = nullptr;
    int* d_first = nullptr;
    std::vector<int> n_search, blocks_search, n_eval, blocks_eval;
    int points_per_block = 4096;
    // lane-mapping threshold (voxels of chunk reach) of the sequences whose
    // mapping is automatic; <= 0: each volume's default
    float pm_threshold = 0.0f;
    // graph
    bool use_graph = false;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches_per_step = 0;
    // autotuner scratch: search states and records
    SearchState* tune_state = nullptr;
    pf_track_stats* tune_stats = nullptr;

    double* rel(int i) const { return poses + 64 * (size_t)i; }
    double* pose(int i) const { return poses + 64 * (size_t)i + 16; }
    double* init(int i) const { return poses + 64 * (size_t)i + 32; }
};

namespace {

int resolve_layout(const pf_volume* v) { return resolve_fitness_layout(v); }

float mapping_threshold(const pf_volume* v, int layout)
{
    const int mapping = (v->fitness_variant >> 2) & 3;
    return mapping == 1 ? -1.0f : mapping == 2 ? INFINITY
                                               : (layout == 3 ? kParticleLanesBelowCells : kParticleLanesBelowNodes);
}

// Point tiles of one problem in a batched launch: about points_per_block
// evaluated points per CTA (work per CTA alike across problems of unequal
// size); a single-pose evaluation spreads over up to 8 CTAs per SM.
int batch_tiles(const pf_batch* b, int K, long long ne_max)
{
    const long long max_tiles = std::max(1LL, (ne_max + SUBTILE - 1) / SUBTILE);
    long long t = K == 1 ? (long long)device_sms(b->device) * 8 : (ne_max + b->points_per_block - 1) / b->points_per_block;
    return (int)std::max(1LL, std::min(t, max_tiles));
}

FitArgs batch_args(const pf_batch* b, int i, SearchState* st, pf_track_stats* stats)
{
    const pf_volume* v = b->vols[i];
    const pf_track_params& p = b->params[i];
    FitArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = v->ws.points;
    a.n_dev = v->ws.n_points;
    a.templ = p.templates_dev;
    a.st = st;
    a.compose_mode = p.compose_mode;
    a.update_mode = p.update_mode;
    a.beta = p.beta;
    a.min_valid_frac = p.min_valid_frac;
    fill_volume_args(a, v);
    a.part_S = v->ws.part_S;
    a.part_C = v->ws.part_C;
    a.counter = v->ws.counter;
    a.stats = stats;
    a.pm_threshold = mapping_threshold(v, b->layout);
    if (b->pm_threshold > 0.0f && ((v->fitness_variant >> 2) & 3) == 0) a.pm_threshold = b->pm_threshold;
    return a;
}

// Builds and uploads the launch tables.  tune: only iteration 0's search,
// on the tuning states (used by the autotuner).
pf_status batch_tables(pf_batch* b, bool tune)
{
    const int n = b->n, iters = b->max_iters;
    // partial slots each volume needs over all iterations, grown first (a
    // reallocation would leave stale pointers in earlier table entries)
    for (int i = 0; i < n; ++i) {
        const pf_track_params& p = b->params[i];
        const long long npix = (long long)b->intrs[i].width * b->intrs[i].height;
        size_t need = 0;
        for (int it = 0; it < p.n_iters; ++it) {
            const int stride = p.decim_sched[it % 3];
            const long long ne_max = (npix + stride - 1) / stride;
            need = std::max(need, (size_t)batch_tiles(b, p.k_sched[it % 3], ne_max) * p.k_sched[it % 3]);
            need = std::max(need, (size_t)batch_tiles(b, 1, ne_max));
        }
        pf_status st = grow_partials(b->vols[i], need);
        if (st != PF_OK) return st;
    }
    std::vector<FitArgs> args((size_t)iters * 2 * n);
    std::vector<int> first((size_t)iters * 2 * (n + 1), 0);
    b->n_search.assign(iters, 0);
    b->blocks_search.assign(iters, 0);
    b->n_eval.assign(iters, 0);
    b->blocks_eval.assign(iters, 0);
    for (int it = 0; it < iters; ++it) {
        for (int kind = 0; kind < 2; ++kind) {
            int cnt = 0, blocks = 0;
            FitArgs* A = args.data() + ((size_t)it * 2 + kind) * n;
            int* F = first.data() + ((size_t)it * 2 + kind) * (n + 1);
            for (int i = 0; i < n; ++i) {
                const pf_track_params& p = b->params[i];
                if (it >= p.n_iters || (tune && (it > 0 || kind == 1))) continue;
                if (kind == 1 && p.update_mode != 0) continue;
                const int K = kind == 0 ? p.k_sched[it % 3] : 1;
                const int stride = p.decim_sched[it % 3];
                const long long npix = (long long)b->intrs[i].width * b->intrs[i].height;
                const long long ne_max = (npix + stride - 1) / stride;
                FitArgs a = tune ? batch_args(b, i, b->tune_state + i, b->tune_stats + i)
                                 : batch_args(b, i, reinterpret_cast<SearchState*>(b->vols[i]->ws.state),
                                              b->stats + i);
                a.K = K;
                a.stride = stride;
                a.iter = it;
                a.n_ptiles = batch_tiles(b, K, ne_max);
                A[cnt] = a;
                F[cnt] = blocks;
                blocks += ((K + KC - 1) / KC) * a.n_ptiles;
                ++cnt;
            }
            F[cnt] = blocks;
            (kind == 0 ? b->n_search : b->n_eval)[it] = cnt;
            (kind == 0 ? b->blocks_search : b->blocks_eval)[it] = blocks;
        }
    }
    if (!b->d_args) {
        PF_CUDA(pf::dev_malloc(&b->d_args, args.size() * sizeof(FitArgs)));
        PF_CUDA(pf::dev_malloc(&b->d_first, first.size() * sizeof(int)));
    }
    PF_CUDA(cudaMemcpy(b->d_args, args.data(), args.size() * sizeof(FitArgs), cudaMemcpyHostToDevice));
    PF_CUDA(cudaMemcpy(b->d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice));
    return PF_OK;
}

template <int SRC, typename TS>
void launch_batch_t(const pf_batch* b, const FitArgs* args, const int* first, int n, int blocks, cudaStream_t s)
{
    if (b->layout == 2)
        fitness_kernel_batch<SRC, 0, TS><<<blocks, FIT_THREADS, 0, s>>>(args, first, n);
    else
        fitness_kernel_batch<SRC, 2, TS><<<blocks, FIT_THREADS, 0, s>>>(args, first, n);
}

template <int SRC>
void launch_batch(const pf_batch* b, int it, int kind, cudaStream_t s)
{
    const int n = kind == 0 ? b->n_search[it] : b->n_eval[it];
    const int blocks = kind == 0 ? b->blocks_search[it] : b->blocks_eval[it];
    if (n == 0) return;
    const FitArgs* args = b->d_args + ((size_t)it * 2 + kind) * b->n;
    const int* first = b->d_first + ((size_t)it * 2 + kind) * (b->n + 1);
    if (b->dtype == PF_F16)
        launch_batch_t<SRC, __half>(b, args, first, n, blocks, s);
    else if (b->dtype == PF_BF16)
        launch_batch_t<SRC, __nv_bfloat16>(b, args, first, n, blocks, s);
    else if (b->dtype == PF_FP8E4M3)
        launch_batch_t<SRC, __nv_fp8_e4m3>(b, args, first, n, blocks, s);
    else
        launch_batch_t<SRC, float>(b, args, first, n, blocks, s);
    pf::count_launch();
}

// One frame of every sequence: compose the initial pose, back-project,
// search (one launch per iteration for all sequences), record the result,
// fuse.
pf_status batch_enqueue(pf_batch* b, cudaStream_t s)
{
    for (int i = 0; i < b->n; ++i) {
        pf_status st = pf_pose_compose(b->pose(i), b->rel(i), b->init(i), s);
        if (st != PF_OK) return st;
        pf_volume* v = b->vols[i];
        track_begin_kernel<<<1, 32, 0, s>>>(reinterpret_cast<SearchState*>(v->ws.state), b->init(i),
                                            b->params[i].init_rot_deg, b->params[i].init_trans_cm, b->stats + i);
        pf::count_launch();
        st = enqueue_backproject(b->depth + b->depth_off[i], &b->intrs[i], v->ws.points, v->ws.block_counts,
                                 v->ws.n_points, s);
        if (st != PF_OK) return st;
    }
    for (int it = 0; it < b->max_iters; ++it) {
        launch_batch<SRC_SEARCH>(b, it, 0, s);
        launch_batch<SRC_EVAL>(b, it, 1, s);
    }
    PF_LAUNCHED();
    for (int i = 0; i < b->n; ++i) {
        pf_volume* v = b->vols[i];
        track_end_kernel<<<1, 32, 0, s>>>(reinterpret_cast<const SearchState*>(v->ws.state), v->ws.n_points,
                                          b->pose(i), b->stats + i);
        pf::count_launch();
        pf_status st = pf_integrate_async(v, b->depth + b->depth_off[i], &b->intrs[i], b->pose(i), s);
        if (st != PF_OK) return st;
    }
    PF_LAUNCHED();
    return PF_OK;
}

void batch_drop_graph(pf_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

}  // namespace

extern "C" {

pf_status pf_batch_create(int n, pf_volume* const* vols, const pf_intrinsics* intrs, const pf_track_params* params,
                          int use_graph, pf_batch** out)
{
    if (!out) return PF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || n > 4096 || !vols || !intrs || !params) return PF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!vols[i]) return PF_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (vols[j] == vols[i]) return PF_ERR_INVALID_ARG;  // a volume holds one sequence's state
        pf_status st = pf::check_intrinsics(intrs + i);
        if (st != PF_OK) return st;
        st = check_params(params + i);
        if (st != PF_OK) return st;
        if (vols[i]->device != vols[0]->device) return PF_ERR_INVALID_ARG;
        const int layout = resolve_layout(vols[i]);
        if (layout == 1 || layout != resolve_layout(vols[0])) return PF_ERR_UNSUPPORTED;
        if (pf_fitness_dtype(vols[i], layout) != pf_fitness_dtype(vols[0], layout)) return PF_ERR_UNSUPPORTED;
    }
    pf_batch* b = new pf_batch();
    b->n = n;
    b->vols.assign(vols, vols + n);
    b->intrs.assign(intrs, intrs + n);
    b->params.assign(params, params + n);
    b->layout = resolve_layout(vols[0]);
    b->dtype = pf_fitness_dtype(vols[0], b->layout);
    b->device = vols[0]->device;
    b->use_graph = use_graph != 0;
    size_t depth_total = 0;
    for (int i = 0; i < n; ++i) {
        b->max_iters = std::max(b->max_iters, params[i].n_iters);
        b->depth_off.push_back(depth_total);
        depth_total += ((size_t)intrs[i].width * intrs[i].height + 63) / 64 * 64;
    }
    auto fail = [&](pf_status st) {
        pf_batch_destroy(b);
        return st;
    };
    pf_status st = PF_OK;
    for (int i = 0; i < n && st == PF_OK; ++i) {
        pf_workspace& w = vols[i]->ws;
        st = pf::workspace_reserve(vols[i], std::max(intrs[i].width * intrs[i].height, w.pix_cap),
                                   std::max(params[i].k_max, w.k_cap));
    }
    if (st != PF_OK) return fail(st);
    cudaError_t e = pf::dev_malloc(&b->depth, depth_total * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(b->depth, 0, depth_total * sizeof(float));
    if (e == cudaSuccess) e = pf::dev_malloc(&b->poses, (size_t)n * 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(b->poses, 0, (size_t)n * 64 * sizeof(double));
    if (e == cudaSuccess) e = pf::dev_malloc(&b->stats, (size_t)n * sizeof(pf_track_stats));
    if (e == cudaSuccess) e = cudaMemset(b->stats, 0, (size_t)n * sizeof(pf_track_stats));
    if (e == cudaSuccess) e = pf::dev_malloc(&b->tune_state, (size_t)n * sizeof(SearchState));
    if (e == cudaSuccess) e = pf::dev_malloc(&b->tune_stats, (size_t)n * sizeof(pf_track_stats));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(pf::cuda_status(e));
    // identity poses
    std::vector<double> I((size_t)n * 64, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 4; ++k)
            for (int q = 0; q < 4; ++q) I[64 * (size_t)i + 16 * k + 5 * q] = 1.0;
    e = cudaMemcpy(b->poses, I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(pf::cuda_status(e));
    st = batch_tables(b, false);
    if (st != PF_OK) return fail(st);
    *out = b;
    return PF_OK;
}

pf_status pf_batch_destroy(pf_batch* b)
{
    if (!b) return PF_OK;
    cudaDeviceSynchronize();
    batch_drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->depth);
    cudaFree(b->poses);
    cudaFree(b->stats);
    cudaFree(b->d_args);
    cudaFree(b->d_first);
    cudaFree(b->tune_state);
    cudaFree(b->tune_stats);
    delete b;
    return PF_OK;
}

pf_status pf_batch_buffers(pf_batch* b, int i, float** depth_dev, double** rel_pose_dev, double** pose_dev,
                           pf_track_stats** stats_dev)
{
    if (!b || i < 0 || i >= b->n) return PF_ERR_INVALID_ARG;
    if (depth_dev) *depth_dev = b->depth + b->depth_off[i];
    if (rel_pose_dev) *rel_pose_dev = b->rel(i);
    if (pose_dev) *pose_dev = b->pose(i);
    if (stats_dev) *stats_dev = b->stats + i;
    return PF_OK;
}

pf_status pf_batch_fuse(pf_batch* b, void* stream)
{
    if (!b) return PF_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) {
        pf_status st = pf_integrate_async(b->vols[i], b->depth + b->depth_off[i], &b->intrs[i], b->pose(i), stream);
        if (st != PF_OK) return st;
    }
    return PF_OK;
}

pf_status pf_batch_step(pf_batch* b, void* stream)
{
    if (!b) return PF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->use_graph) return batch_enqueue(b, s);
    if (!b->exec) {
        const bool timing = pf::timing_swap(false);
        const unsigned long long c0 = pf::g_launches.load();
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        pf_status st = e == cudaSuccess ? batch_enqueue(b, b->cap) : pf::cuda_status(e);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
        const unsigned long long c1 = pf::g_launches.load();
        pf::g_launches.fetch_sub(c1 - c0);
        pf::timing_swap(timing);
        if (st == PF_OK && e2 != cudaSuccess) st = pf::cuda_status(e2);
        if (st != PF_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        b->graph = g;
        b->launches_per_step = c1 - c0;
        PF_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    PF_CUDA(cudaGraphLaunch(b->exec, s));
    pf::count_launch((unsigned)b->launches_per_step);
    return PF_OK;
}

pf_status pf_batch_set_points_per_block(pf_batch* b, int points_per_block)
{
    if (!b || points_per_block < SUBTILE || points_per_block > (1 << 24)) return PF_ERR_INVALID_ARG;
    PF_CUDA(cudaDeviceSynchronize());
    b->points_per_block = points_per_block;
    batch_drop_graph(b);
    return batch_tables(b, false);
}

pf_status pf_batch_set_mapping_threshold(pf_batch* b, float voxels)
{
    if (!b || !(voxels <= 1e6f)) return PF_ERR_INVALID_ARG;
    PF_CUDA(cudaDeviceSynchronize());
    b->pm_threshold = voxels > 0.0f ? voxels : 0.0f;
    batch_drop_graph(b);
    return batch_tables(b, false);
}

pf_status pf_batch_tuning(const pf_batch* b, int* points_per_block, float* mapping_threshold)
{
    if (!b) return PF_ERR_INVALID_ARG;
    if (points_per_block) *points_per_block = b->points_per_block;
    if (mapping_threshold) *mapping_threshold = b->pm_threshold;
    return PF_OK;
}

// The autotuner's two axes, tuned one after the other on copies of the
// search state (the first search iteration of the current frames):
//   1. points per CTA of the batched launches, timed at the initial search
//      size (lanes on points) and at 1e-3 of it (lanes on particles),
//      weights 1 : 3 (about the two regimes' shares of a 20-iteration search);
//   2. the lane-mapping threshold (voxels of a particle chunk's reach below
//      which particles take the lanes), timed at search sizes 0.3, 0.1 and
//      0.03 of the initial one, where chunks cross from one mapping to the
//      other.
// Each timing is the second of two runs (the first warms up).
pf_status pf_batch_autotune(pf_batch* b, void* stream, int* chosen)
{
    if (!b) return PF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < b->n; ++i) {
        pf_volume* v = b->vols[i];
        pf_status st = enqueue_backproject(b->depth + b->depth_off[i], &b->intrs[i], v->ws.points,
                                           v->ws.block_counts, v->ws.n_points, s);
        if (st != PF_OK) return st;
    }
    cudaEvent_t e0, e1;
    PF_CUDA(cudaEventCreate(&e0));
    PF_CUDA(cudaEventCreate(&e1));
    pf_status st = PF_OK;
    // total time of the first search iteration at the given search-size
    // scales and weights, for the current tables
    auto time_regimes = [&](const double* scale, const float* weight, int n_regimes, float& total) {
        total = 0.0f;
        for (int regime = 0; regime < n_regimes && st == PF_OK; ++regime) {
            for (int rep = 0; rep < 2; ++rep) {
                for (int i = 0; i < b->n; ++i)
                    track_begin_kernel<<<1, 32, 0, s>>>(b->tune_state + i, b->pose(i),
                                                        b->params[i].init_rot_deg * scale[regime],
                                                        b->params[i].init_trans_cm * scale[regime], b->tune_stats + i);
                cudaEventRecord(e0, s);
                launch_batch<SRC_SEARCH>(b, 0, 0, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = PF_ERR_CUDA;
                    return;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1) total += weight[regime] * ms;
            }
        }
    };
    const int saved = b->points_per_block;
    const float saved_pm = b->pm_threshold;
    int best = saved;
    float best_ms = INFINITY;
    const int candidates[] = {1024, 2048, 4096, 8192, 16384, 32768, 65536, 131072};
    const double scale1[2] = {1.0, 1e-3};
    const float weight1[2] = {1.0f, 3.0f};
    for (int c : candidates) {
        b->points_per_block = c;
        st = batch_tables(b, true);
        if (st != PF_OK) break;
        float total = 0.0f;
        time_regimes(scale1, weight1, 2, total);
        if (st != PF_OK) break;
        if (total < best_ms) {
            best_ms = total;
            best = c;
        }
    }
    b->points_per_block = st == PF_OK ? best : saved;
    float best_pm = saved_pm;
    if (st == PF_OK) {
        const float thresholds[] = {0.0f, 2.0f, 3.0f, 8.0f, 12.0f, 20.0f};  // 0: each volume's default
        const double scale2[3] = {0.3, 0.1, 0.03};
        const float weight2[3] = {1.0f, 1.0f, 1.0f};
        float best_t = INFINITY;
        for (float t : thresholds) {
            b->pm_threshold = t;
            st = batch_tables(b, true);
            if (st != PF_OK) break;
            float total = 0.0f;
            time_regimes(scale2, weight2, 3, total);
            if (st != PF_OK) break;
            if (total < best_t) {
                best_t = total;
                best_pm = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PF_OK) b->points_per_block = saved;
    b->pm_threshold = st == PF_OK ? best_pm : saved_pm;
    batch_drop_graph(b);
    pf_status st2 = batch_tables(b, false);
    if (chosen) *chosen = b->points_per_block;
    return st != PF_OK ? st : st2;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fitness without any device allocation.
//
// pf_fitness keeps its per-tile partial sums in the volume's workspace and
// grows it with cudaMalloc when a call needs more.  Callers that must not
// allocate device memory once they are running -- for instance a process
// whose device memory is owned by another allocator, or a real-time loop
// that cannot afford the device-wide synchronisation a cudaMalloc implies --
// use pf_fitness_noalloc instead: the same kernel, with its scratch (the
// partial sums and the ticket counter of the last-block reduction) in the
// fixed array below, which every device that loads the library holds until
// the process exits.
// ---------------------------------------------------------------------------
namespace {

struct NoAllocScratch {
    unsigned int counter;              // ticket counter; must be zero when a launch starts
    unsigned int pad[63];
    float S[PF_NOALLOC_MAX_SLOTS];     // partial sums, one per (point tile, pose)
    int C[PF_NOALLOC_MAX_SLOTS];       // partial counts
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
NoAllocScratch* g_noalloc_addr[kMaxDevices] = {};

// Loads the code of every fitness kernel pf_fitness_noalloc can launch (each
// layout and storage type) on the current device.  With lazy module loading,
// a kernel's code is loaded -- into newly allocated device memory -- on its
// first launch; doing it here, in the set-up, keeps later calls free of
// allocations whatever volume they are given.
template <typename TS>
cudaError_t preload_fitness_storage()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fitness_kernel<SRC_POSES, 0, TS>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fitness_kernel<SRC_POSES, 2, TS>);
    return e;
}

cudaError_t preload_fitness_kernels()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fitness_kernel<SRC_POSES, 1, float>);
    if (e == cudaSuccess) e = preload_fitness_storage<float>();
    if (e == cudaSuccess) e = preload_fitness_storage<__half>();
    if (e == cudaSuccess) e = preload_fitness_storage<__nv_bfloat16>();
    if (e == cudaSuccess) e = preload_fitness_storage<__nv_fp8_e4m3>();
    return e;
}

// Device address of the scratch array on the current device, which must be
// `device`.  The first call on a device is the set-up: it looks the address
// up and loads the kernels (both may allocate); later calls only read the
// cached address.
pf_status noalloc_scratch(int device, NoAllocScratch** out)
{
    int dev = 0;
    PF_CUDA(cudaGetDevice(&dev));
    if (dev != device) return PF_ERR_INVALID_ARG;  // the array and the volume would be on different devices
    if (dev < 0 || dev >= kMaxDevices) return PF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return pf::cuda_status(e);
        if (!p) return PF_ERR_CUDA;
        e = preload_fitness_kernels();
        if (e != cudaSuccess) return pf::cuda_status(e);
        g_noalloc_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_noalloc_addr[dev];
    return PF_OK;
}

}  // namespace

static pf_status pf_fitness_noalloc_impl(const pf_volume* v, const float* points_dev, int n, const float* poses_dev,
                                         int k, float* fitness_dev, int* count_dev, void* stream)
{
    if (!v || !poses_dev || !fitness_dev || !count_dev) return PF_ERR_INVALID_ARG;
    if (n < 0 || k < 1 || (n > 0 && !points_dev)) return PF_ERR_INVALID_ARG;
    if (k > PF_NOALLOC_MAX_SLOTS) return PF_ERR_INVALID_ARG;  // more poses than the scratch holds
    NoAllocScratch* sc = nullptr;
    pf_status st = noalloc_scratch(v->device, &sc);
    if (st != PF_OK) return st;
    const int chunks = (k + KC - 1) / KC;
    // as many point tiles as pf_fitness would use, within the fixed scratch
    const int tiles = std::max(1, std::min(choose_ptiles(v->device, chunks, n), PF_NOALLOC_MAX_SLOTS / k));
    FitArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = reinterpret_cast<const float4*>(points_dev);
    a.n_dev = nullptr;
    a.n_host = n;
    a.stride = 1;
    a.K = k;
    a.poses = poses_dev;
    fill_volume_args(a, v);
    a.part_S = sc->S;
    a.part_C = sc->C;
    a.counter = &sc->counter;
    a.n_ptiles = tiles;
    a.out_E = fitness_dev;
    a.out_C = count_dev;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the counter must start at zero
    PF_CUDA(cudaMemsetAsync(&sc->counter, 0, sizeof(unsigned int), s));
    launch_fitness<SRC_POSES>(a, v->fitness_variant, v, chunks, s);
    PF_LAUNCHED();
    return PF_OK;
}

// Every entry point that takes a volume keeps its last failing status
// there (pf_volume_last_error).
extern "C" {

pf_status pf_fitness(const pf_volume* cv, const float* points_dev, int n, const float* poses_dev, int k,
                     float* fitness_dev, int* count_dev, void* stream)
{
    return pf::keep_status(cv, pf_fitness_impl(cv, points_dev, n, poses_dev, k, fitness_dev, count_dev, stream));
}

pf_status pf_track_reserve(pf_volume* v, int max_pixels, int k_max)
{
    return pf::keep_status(v, pf_track_reserve_impl(v, max_pixels, k_max));
}

pf_status pf_track_frame_async(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr,
                               const pf_track_params* p, const double* init_pose_dev, double* out_pose_dev,
                               pf_track_stats* stats_dev, void* stream)
{
    return pf::keep_status(v, pf_track_frame_async_impl(v, depth_dev, intr, p, init_pose_dev, out_pose_dev, stats_dev,
                                                        stream));
}

pf_status pf_track_frame(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr, const pf_track_params* p,
                         const double init_pose[16], double out_pose[16], pf_track_stats* stats_host, void* stream)
{
    return pf::keep_status(v, pf_track_frame_impl(v, depth_dev, intr, p, init_pose, out_pose, stats_host, stream));
}

pf_status pf_fitness_noalloc(const pf_volume* v, const float* points_dev, int n, const float* poses_dev, int k,
                             float* fitness_dev, int* count_dev, void* stream)
{
    return pf::keep_status(v, pf_fitness_noalloc_impl(v, points_dev, n, poses_dev, k, fitness_dev, count_dev,
                                                      stream));
}

}  // extern "C"
