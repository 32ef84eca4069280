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
//     fixed order -- no floating-point atomics, bit-reproducible.
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

#include "pf_internal.cuh"

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
// ---------------------------------------------------------------------------
constexpr int BP_THREADS = 256, BP_PPT = 8, BP_CHUNK = BP_THREADS * BP_PPT;

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

__global__ void __launch_bounds__(BP_THREADS) bp_count_kernel(const float* __restrict__ depth, int npix,
                                                              float dmin, float dmax, int* block_counts)
{
    __shared__ int sh[32];
    const int base = blockIdx.x * BP_CHUNK + threadIdx.x * BP_PPT;
    int c = 0;
#pragma unroll
    for (int p = 0; p < BP_PPT; ++p) {
        const int idx = base + p;
        if (idx < npix && pf_depth_usable(depth[idx], dmin, dmax)) ++c;
    }
    const int tot = block_sum_int(c, sh);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(BP_THREADS) bp_write_kernel(const float* __restrict__ depth, CamK cam,
                                                              int npix, const int* __restrict__ block_counts,
                                                              float4* __restrict__ pts, int* n_out)
{
    __shared__ int sh[32];
    __shared__ int warp_off[32];
    // points of the earlier chunks
    int off = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) off += block_counts[b];
    off = block_sum_int(off, sh);

    const int base = blockIdx.x * BP_CHUNK + threadIdx.x * BP_PPT;
    float z[BP_PPT];
    int c = 0;
#pragma unroll
    for (int p = 0; p < BP_PPT; ++p) {
        const int idx = base + p;
        z[p] = idx < npix ? depth[idx] : 0.0f;
        if (idx < npix && pf_depth_usable(z[p], cam.dmin, cam.dmax)) ++c;
        else z[p] = NAN;
    }
    // exclusive scan of c over the block, in thread order (= pixel order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_off[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            int t = warp_off[w];
            warp_off[w] = acc;
            acc += t;
        }
    }
    __syncthreads();
    int pos = off + warp_off[warp] + incl - c;
#pragma unroll
    for (int p = 0; p < BP_PPT; ++p) {
        if (z[p] == z[p]) {
            const int idx = base + p;
            const int v = idx / cam.width, u = idx - v * cam.width;
            const float zz = z[p];
            const float x = __fdiv_rn(((float)u - cam.cx) * zz, cam.fx);
            const float y = __fdiv_rn(((float)v - cam.cy) * zz, cam.fy);
            pts[pos++] = make_float4(x, y, zz, 0.0f);
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *n_out = pos;
}

pf_status enqueue_backproject(const float* depth, const pf_intrinsics* intr, float4* pts, int* block_counts,
                              int* n_out, cudaStream_t s)
{
    const int npix = intr->width * intr->height;
    const int blocks = (npix + BP_CHUNK - 1) / BP_CHUNK;
    CamK cam = make_cam(intr);
    pf::timing_begin(pf::KC_BACKPROJECT, s);
    bp_count_kernel<<<blocks, BP_THREADS, 0, s>>>(depth, npix, cam.dmin, cam.dmax, block_counts);
    bp_write_kernel<<<blocks, BP_THREADS, 0, s>>>(depth, cam, npix, block_counts, pts, n_out);
    pf::count_launch(2);
    pf::timing_end(pf::KC_BACKPROJECT, s);
    PF_LAUNCHED();
    return PF_OK;
}

// ---------------------------------------------------------------------------
// Fitness
// ---------------------------------------------------------------------------
constexpr int FIT_THREADS = 256;
constexpr int FIT_WARPS = FIT_THREADS / 32;
constexpr int KC = 32;    // particles per CTA
constexpr int PPT = 8;    // points per thread per sub-tile
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
    SearchState* st;
    int compose_mode, update_mode;
    double beta;
    float min_valid_frac;
    // volume
    const float* tsdf;
    const float* weight;
    const float4* cells;
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

__device__ inline void so3_exp_d(const double w[3], double R[9])
{
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = sqrt(th2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        double sh = sin(0.5 * th), ch = cos(0.5 * th);
        a = 2.0 * sh * ch / th;
        b = 2.0 * sh * sh / th2;
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

// A particle as the sampling loop uses it.  g = (A_hi + A_lo) x + b maps a
// camera-frame point to grid units relative to an integer cell offset o: the
// grid coordinate is g + o.  A = R / voxel carried as a float pair and
// |b| < 1 make the transform as accurate as the FP64 pose it came from (the
// rounding of a single float matrix would shift every point of a particle
// the same way); the offset is folded into the cell bounds [lo, hi) and into
// the magic constant of the floor, so it costs nothing per sample.
struct Particle {      // shared memory, 128 bytes
    float4 h0, h1, h2; // rows of A_hi | b
    float4 l0, l1, l2; // rows of A_lo | lo bound
    float4 u;          // hi bounds x y z | magic x
    float4 m;          // magic y z | translation, rotation distance to the chunk's first particle
};

struct Xform {         // the same in registers
    float a[9], l[9], b[3], lo[3], hi[3];
    int mg[3];
};

constexpr int kMagicBits = 0x4b400000;  // bits of 1.5 * 2^23

// Grid-unit particle from a camera-to-world pose [R | t] given in FP64.
__device__ inline void make_particle(const double R[9], const double t[3], const FitArgs& a, Particle& P)
{
    const double iv = 1.0 / a.vs;
    const int n[3] = {a.nx, a.ny, a.nz};
    float hi_[3][4], lo_[3][3], lob[3], hib[3];
    int magic[3];
    bool ok = true;
    for (int r = 0; r < 3; ++r) {
        const double tg = (t[r] - a.org[r]) * iv;
        ok = ok && fabs(tg) < 2097152.0;  // 2^21: beyond, no point can reach the grid
        const double o = ok ? floor(tg) : 0.0;
        for (int c = 0; c < 3; ++c) {
            const double Ag = R[3 * r + c] * iv;
            const float h = (float)Ag;
            hi_[r][c] = h;
            lo_[r][c] = (float)(Ag - (double)h);
        }
        hi_[r][3] = (float)(tg - o);
        lob[r] = (float)(-o);
        hib[r] = (float)((double)(n[r] - 1) - o);
        magic[r] = kMagicBits - (int)o;
    }
    if (!ok)
        for (int r = 0; r < 3; ++r) {
            lob[r] = 1.0f;
            hib[r] = 0.0f;
        }
    P.h0 = make_float4(hi_[0][0], hi_[0][1], hi_[0][2], hi_[0][3]);
    P.h1 = make_float4(hi_[1][0], hi_[1][1], hi_[1][2], hi_[1][3]);
    P.h2 = make_float4(hi_[2][0], hi_[2][1], hi_[2][2], hi_[2][3]);
    P.l0 = make_float4(lo_[0][0], lo_[0][1], lo_[0][2], lob[0]);
    P.l1 = make_float4(lo_[1][0], lo_[1][1], lo_[1][2], lob[1]);
    P.l2 = make_float4(lo_[2][0], lo_[2][1], lo_[2][2], lob[2]);
    P.u = make_float4(hib[0], hib[1], hib[2], __int_as_float(magic[0]));
    P.m = make_float4(__int_as_float(magic[1]), __int_as_float(magic[2]), 0.0f, 0.0f);
}

__device__ __forceinline__ void load_xform(const Particle& P, Xform& X)
{
    const float4 h0 = P.h0, h1 = P.h1, h2 = P.h2, l0 = P.l0, l1 = P.l1, l2 = P.l2, u = P.u, m = P.m;
    X.a[0] = h0.x; X.a[1] = h0.y; X.a[2] = h0.z; X.b[0] = h0.w;
    X.a[3] = h1.x; X.a[4] = h1.y; X.a[5] = h1.z; X.b[1] = h1.w;
    X.a[6] = h2.x; X.a[7] = h2.y; X.a[8] = h2.z; X.b[2] = h2.w;
    X.l[0] = l0.x; X.l[1] = l0.y; X.l[2] = l0.z; X.lo[0] = l0.w;
    X.l[3] = l1.x; X.l[4] = l1.y; X.l[5] = l1.z; X.lo[1] = l1.w;
    X.l[6] = l2.x; X.l[7] = l2.y; X.l[8] = l2.z; X.lo[2] = l2.w;
    X.hi[0] = u.x; X.hi[1] = u.y; X.hi[2] = u.z; X.mg[0] = __float_as_int(u.w);
    X.mg[1] = __float_as_int(m.x); X.mg[2] = __float_as_int(m.y);
}

// Grid coordinates (relative to the particle's cell offset) of a point:
// the small A_lo terms and b first, then A_hi.
__device__ __forceinline__ void apply(const Xform& X, float x, float y, float z, float& gx, float& gy, float& gz)
{
    gx = fmaf(X.a[0], x, fmaf(X.a[1], y, fmaf(X.a[2], z, fmaf(X.l[0], x, fmaf(X.l[1], y, fmaf(X.l[2], z, X.b[0]))))));
    gy = fmaf(X.a[3], x, fmaf(X.a[4], y, fmaf(X.a[5], z, fmaf(X.l[3], x, fmaf(X.l[4], y, fmaf(X.l[5], z, X.b[1]))))));
    gz = fmaf(X.a[6], x, fmaf(X.a[7], y, fmaf(X.a[8], z, fmaf(X.l[6], x, fmaf(X.l[7], y, fmaf(X.l[8], z, X.b[2]))))));
}

// Fast-path sample: tsdf only.  Non-finite nodes (unobserved or outside the
// band) make the interpolated value non-finite, so the validity test of the
// cell is a single comparison on the result.
__device__ __forceinline__ void sample_encoded(const float* __restrict__ tsdf, int nx, int nxy, const Xform& X,
                                               float gx, float gy, float gz, float& s, int& c)
{
    if (gx >= X.lo[0] && gx < X.hi[0] && gy >= X.lo[1] && gy < X.hi[1] && gz >= X.lo[2] && gz < X.hi[2]) {
        // floor(g) for |g| < 2^22: adding 1.5*2^23 rounding down leaves
        // floor(g) in the low mantissa bits and keeps every step exact; the
        // particle's magic constant also adds its integer cell offset
        const float M = 12582912.0f;
        const float rx = __fadd_rd(gx, M), ry = __fadd_rd(gy, M), rz = __fadd_rd(gz, M);
        const int ix = __float_as_int(rx) - X.mg[0];
        const int iy = __float_as_int(ry) - X.mg[1];
        const int iz = __float_as_int(rz) - X.mg[2];
        const float fx = gx - (rx - M), fy = gy - (ry - M), fz = gz - (rz - M);
        const float* p = tsdf + (ix + nx * iy + nxy * iz);
        const float v000 = __ldg(p), v100 = __ldg(p + 1);
        const float v010 = __ldg(p + nx), v110 = __ldg(p + nx + 1);
        const float v001 = __ldg(p + nxy), v101 = __ldg(p + nxy + 1);
        const float v011 = __ldg(p + nxy + nx), v111 = __ldg(p + nxy + nx + 1);
        const float x00 = fmaf(fx, v100 - v000, v000);
        const float x10 = fmaf(fx, v110 - v010, v010);
        const float x01 = fmaf(fx, v101 - v001, v001);
        const float x11 = fmaf(fx, v111 - v011, v011);
        const float y0 = fmaf(fy, x10 - x00, x00);
        const float y1 = fmaf(fy, x11 - x01, x01);
        const float t = fabsf(fmaf(fz, y1 - y0, y0));
        if (t < INFINITY) {
            s += t;
            c += 1;
        }
    }
}

// Plain sample: tsdf and weight, all eight nodes tested explicitly.
__device__ __forceinline__ void sample_plain(const float* __restrict__ tsdf, const float* __restrict__ weight, int nx,
                                             int nxy, const Xform& X, float gx, float gy, float gz, float& s, int& c)
{
    if (gx >= X.lo[0] && gx < X.hi[0] && gy >= X.lo[1] && gy < X.hi[1] && gz >= X.lo[2] && gz < X.hi[2]) {
        const float M = 12582912.0f;
        const float rx = __fadd_rd(gx, M), ry = __fadd_rd(gy, M), rz = __fadd_rd(gz, M);
        const int base = (__float_as_int(rx) - X.mg[0]) + nx * (__float_as_int(ry) - X.mg[1]) +
                         nxy * (__float_as_int(rz) - X.mg[2]);
        const float fx = gx - (rx - M), fy = gy - (ry - M), fz = gz - (rz - M);
        const int off[8] = {0, 1, nx, nx + 1, nxy, nxy + 1, nxy + nx, nxy + nx + 1};
        float v[8];
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float w = __ldg(weight + base + off[q]);
            v[q] = __ldg(tsdf + base + off[q]);
            ok = ok && (w > 0.0f) && (fabsf(v[q]) < 1.0f);
        }
        if (ok) {
            const float x00 = fmaf(fx, v[1] - v[0], v[0]);
            const float x10 = fmaf(fx, v[3] - v[2], v[2]);
            const float x01 = fmaf(fx, v[5] - v[4], v[4]);
            const float x11 = fmaf(fx, v[7] - v[6], v[6]);
            const float y0 = fmaf(fy, x10 - x00, x00);
            const float y1 = fmaf(fy, x11 - x01, x01);
            s += fabsf(fmaf(fz, y1 - y0, y0));
            c += 1;
        }
    }
}

// Cell-view sample: the eight corners of the cell are one 32-byte sector,
// fetched as two 16-byte loads; same arithmetic as sample_encoded.
__device__ __forceinline__ void sample_cells(const float4* __restrict__ cells, int nx, int nxy, const Xform& X,
                                             float gx, float gy, float gz, float& s, int& c)
{
    if (gx >= X.lo[0] && gx < X.hi[0] && gy >= X.lo[1] && gy < X.hi[1] && gz >= X.lo[2] && gz < X.hi[2]) {
        const float M = 12582912.0f;
        const float rx = __fadd_rd(gx, M), ry = __fadd_rd(gy, M), rz = __fadd_rd(gz, M);
        const int idx = (__float_as_int(rx) - X.mg[0]) + nx * (__float_as_int(ry) - X.mg[1]) +
                        nxy * (__float_as_int(rz) - X.mg[2]);
        const float fx = gx - (rx - M), fy = gy - (ry - M), fz = gz - (rz - M);
        const float4* p = cells + 2 * (size_t)idx;
        const float4 lo = __ldg(p), hi = __ldg(p + 1);
        const float x00 = fmaf(fx, lo.y - lo.x, lo.x);
        const float x10 = fmaf(fx, lo.w - lo.z, lo.z);
        const float x01 = fmaf(fx, hi.y - hi.x, hi.x);
        const float x11 = fmaf(fx, hi.w - hi.z, hi.z);
        const float y0 = fmaf(fy, x10 - x00, x00);
        const float y1 = fmaf(fy, x11 - x01, x01);
        const float t = fabsf(fmaf(fz, y1 - y0, y0));
        if (t < INFINITY) {
            s += t;
            c += 1;
        }
    }
}

// VARIANT: 0 encoded tsdf nodes, 1 plain (tsdf + weight), 2 cell view.
template <int VARIANT>
__device__ __forceinline__ void sample(const FitArgs& a, int nx, int nxy, const Xform& X, float x, float y, float z,
                                       float& s, int& c)
{
    float gx, gy, gz;
    apply(X, x, y, z, gx, gy, gz);
    if (VARIANT == 0)
        sample_encoded(a.tsdf, nx, nxy, X, gx, gy, gz, s, c);
    else if (VARIANT == 1)
        sample_plain(a.tsdf, a.weight, nx, nxy, X, gx, gy, gz, s, c);
    else
        sample_cells(a.cells, nx, nxy, X, gx, gy, gz, s, c);
}

// Particles k_begin .. k_begin+kc-1 of this launch into shared memory, in FP64
// (the search composes dP_k * P exactly as the pose update does).
template <int SRC>
__device__ void build_particles(const FitArgs& a, int k_begin, int kc, Particle* sP)
{
    const int t = threadIdx.x;
    if (t >= kc) return;
    const int k = k_begin + t;
    double R[9], tw[3];
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
            so3_exp_d(dw, dR);
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c)
                    R[3 * r + c] = dR[3 * r] * P[c] + dR[3 * r + 1] * P[4 + c] + dR[3 * r + 2] * P[8 + c];
                const double tr = a.compose_mode == 0 ? dR[3 * r] * P[3] + dR[3 * r + 1] * P[7] + dR[3 * r + 2] * P[11]
                                                      : P[4 * r + 3];
                tw[r] = tr + wt * (double)u[3 + r];
            }
        }
    }
    make_particle(R, tw, a, sP[t]);
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

template <int SRC, int VARIANT>
__global__ void __launch_bounds__(FIT_THREADS, 3) fitness_kernel(FitArgs a)
{
    __shared__ Particle sP[KC];
    __shared__ float accS[FIT_WARPS][KC];
    __shared__ int accC[FIT_WARPS][KC];
    __shared__ int s_last;
    __shared__ int s_skip;
    __shared__ int s_mode;
    __shared__ float s_spread[2];
    __shared__ float s_red[FIT_WARPS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k_begin = blockIdx.x * KC;
    const int kc = min(KC, a.K - k_begin);

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
    if (!skip) build_particles<SRC>(a, k_begin, kc, sP);
    __syncthreads();
    // spread of the chunk's particles: translation (voxels) and rotation
    // (voxels per metre) relative to its first particle
    if (tid == 0) {
        float dt = 0.0f, dr = 0.0f;
        if (!skip) {
            const Particle& P0 = sP[0];
            const float o0[3] = {(float)(kMagicBits - __float_as_int(P0.u.w)), (float)(kMagicBits - __float_as_int(P0.m.x)),
                                 (float)(kMagicBits - __float_as_int(P0.m.y))};
            for (int k = 1; k < kc; ++k) {
                const Particle& P = sP[k];
                const float ok_[3] = {(float)(kMagicBits - __float_as_int(P.u.w)), (float)(kMagicBits - __float_as_int(P.m.x)),
                                      (float)(kMagicBits - __float_as_int(P.m.y))};
                dt = fmaxf(dt, fabsf((ok_[0] + P.h0.w) - (o0[0] + P0.h0.w)));
                dt = fmaxf(dt, fabsf((ok_[1] + P.h1.w) - (o0[1] + P0.h1.w)));
                dt = fmaxf(dt, fabsf((ok_[2] + P.h2.w) - (o0[2] + P0.h2.w)));
                dr = fmaxf(dr, fabsf(P.h0.x - P0.h0.x) + fabsf(P.h0.y - P0.h0.y) + fabsf(P.h0.z - P0.h0.z));
                dr = fmaxf(dr, fabsf(P.h1.x - P0.h1.x) + fabsf(P.h1.y - P0.h1.y) + fabsf(P.h1.z - P0.h1.z));
                dr = fmaxf(dr, fabsf(P.h2.x - P0.h2.x) + fabsf(P.h2.y - P0.h2.y) + fabsf(P.h2.z - P0.h2.z));
            }
        }
        s_spread[0] = dt;
        s_spread[1] = dr;
    }
    __syncthreads();

    const int N = a.n_dev ? *a.n_dev : a.n_host;
    const long long Ne = N > 0 ? ((long long)N + a.stride - 1) / a.stride : 0;
    const long long beg = Ne * blockIdx.y / a.n_ptiles;
    const long long end = Ne * (blockIdx.y + 1) / a.n_ptiles;
    const int nx = a.nx, nxy = a.nx * a.ny;

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
            // mapping of this sub-tile: when every particle puts a point in
            // (nearly) the same cell, lanes take particles and share a point,
            // so each gather of a warp touches one or two sectors; otherwise
            // lanes take neighbouring image points of one particle
            for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
            if (lane == 0) s_red[warp] = r2;
            __syncthreads();
            if (tid == 0) {
                float m = 0.0f;
                for (int w = 0; w < FIT_WARPS; ++w) m = fmaxf(m, s_red[w]);
                // (a chunk of fewer than 24 particles would leave lanes idle)
                s_mode = kc >= 24 && (s_spread[0] + s_spread[1] * sqrtf(m)) < a.pm_threshold;
            }
            __syncthreads();
            if (!s_mode) {
                for (int kk = 0; kk < kc; ++kk) {
                    Xform X;
                    load_xform(sP[kk], X);
                    float s = 0.0f;
                    int c = 0;
#pragma unroll
                    for (int p = 0; p < PPT; ++p) sample<VARIANT>(a, nx, nxy, X, px[p], py[p], pz[p], s, c);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        s += __shfl_xor_sync(0xffffffffu, s, o);
                        c += __shfl_xor_sync(0xffffffffu, c, o);
                    }
                    if (lane == 0) {
                        accS[warp][kk] += s;
                        accC[warp][kk] += c;
                    }
                }
            } else {
                Xform X;
                load_xform(sP[lane < kc ? lane : 0], X);
                float s = 0.0f;
                int c = 0;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    for (int j = 0; j < 32; ++j) {
                        const float x = __shfl_sync(0xffffffffu, px[p], j);
                        const float y = __shfl_sync(0xffffffffu, py[p], j);
                        const float z = __shfl_sync(0xffffffffu, pz[p], j);
                        sample<VARIANT>(a, nx, nxy, X, x, y, z, s, c);
                    }
                }
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
        const size_t slot = (size_t)blockIdx.y * a.K + k_begin + tid;
        a.part_S[slot] = S;
        a.part_C[slot] = C;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int ticket = atomicAdd(a.counter, 1u);
        s_last = ticket == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ------------------------------------------------------------------
    // Last CTA: reduce partials over point tiles (fixed order) and finish.
    // ------------------------------------------------------------------
    if (SRC == SRC_POSES) {
        for (int k = tid; k < a.K; k += FIT_THREADS) {
            float S = 0.0f;
            int C = 0;
            for (int y = 0; y < a.n_ptiles; ++y) {
                S += __ldcg(a.part_S + (size_t)y * a.K + k);
                C += __ldcg(a.part_C + (size_t)y * a.K + k);
            }
            a.out_E[k] = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
            a.out_C[k] = C;
        }
    } else if (SRC == SRC_EVAL) {
        if (tid == 0) {
            if (!skip) {
                float S = 0.0f;
                int C = 0;
                for (int y = 0; y < a.n_ptiles; ++y) {
                    S += __ldcg(a.part_S + y);
                    C += __ldcg(a.part_C + y);
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
            float S = 0.0f;
            int C = 0;
            for (int y = 0; y < a.n_ptiles; ++y) {
                S += __ldcg(a.part_S + (size_t)y * a.K);
                C += __ldcg(a.part_C + (size_t)y * a.K);
            }
            s_E0 = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
            s_C0 = C;
        }
        __syncthreads();
        const float E0 = s_E0;
        float be = INFINITY;
        int bk = 0x7fffffff;
        int nadv = 0;
        double sum[6] = {0, 0, 0, 0, 0, 0};
        for (int k = tid; k < a.K; k += FIT_THREADS) {
            float S = 0.0f;
            int C = 0;
            for (int y = 0; y < a.n_ptiles; ++y) {
                S += __ldcg(a.part_S + (size_t)y * a.K + k);
                C += __ldcg(a.part_C + (size_t)y * a.K + k);
            }
            const float E = C > 0 ? __fdiv_rn(S, (float)C) : INFINITY;
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

// Point tiles for a launch with `chunks` particle chunks over at most
// `ne_max` evaluated points: enough CTAs for about two full waves.
int choose_ptiles(int dev, int chunks, long long ne_max)
{
    const long long target = (long long)device_sms(dev) * 4 * 2;
    long long tiles = (target + chunks - 1) / chunks;
    const long long max_tiles = std::max(1LL, (ne_max + SUBTILE - 1) / SUBTILE);
    tiles = std::min(tiles, max_tiles);
    return (int)std::max(1LL, tiles);
}

// variant = layout + 4 * mapping (see pf_set_fitness_variant).  Measured on
// the 640x480 / 512^3 workload, particles on lanes win below a spread of
// about 0.5 degree and 0.5 cm with the cell view (~5 voxels by the bound
// used here) and below about 1 degree and 1 cm on the node array (~12).
constexpr float kParticleLanesBelowCells = 5.0f;
constexpr float kParticleLanesBelowNodes = 12.0f;

template <int SRC>
void launch_fitness(FitArgs a, int variant, bool has_cells, int chunks, cudaStream_t s)
{
    const int mapping = (variant >> 2) & 3;
    int layout = variant & 3;
    if (layout == 0) layout = has_cells ? 3 : 2;
    const float auto_threshold = layout == 3 ? kParticleLanesBelowCells : kParticleLanesBelowNodes;
    a.pm_threshold = mapping == 1 ? -1.0f : mapping == 2 ? INFINITY : auto_threshold;
    dim3 grid(chunks, a.n_ptiles);
    if (layout == 2)
        fitness_kernel<SRC, 0><<<grid, FIT_THREADS, 0, s>>>(a);
    else if (layout == 1)
        fitness_kernel<SRC, 1><<<grid, FIT_THREADS, 0, s>>>(a);
    else
        fitness_kernel<SRC, 2><<<grid, FIT_THREADS, 0, s>>>(a);
    pf::count_launch();
}

void fill_volume_args(FitArgs& a, const pf_volume* v)
{
    a.tsdf = v->tsdf;
    a.weight = v->weight;
    a.cells = v->cells;
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
        PF_CUDA(cudaMalloc(&w.counter, sizeof(unsigned int)));
        PF_CUDA(cudaMemset(w.counter, 0, sizeof(unsigned int)));
    }
    if ((size_t)w.part_cap < need) {
        cudaFree(w.part_S);
        cudaFree(w.part_C);
        w.part_S = nullptr;
        w.part_C = nullptr;
        w.part_cap = 0;
        PF_CUDA(cudaMalloc(&w.part_S, need * sizeof(float)));
        PF_CUDA(cudaMalloc(&w.part_C, need * sizeof(int)));
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
    // up to k_max (decimation only lowers the number of tiles)
    size_t need = 0;
    for (int chunks = 1; chunks <= (k_max + KC - 1) / KC; ++chunks) {
        const size_t K = std::min((size_t)chunks * KC, (size_t)k_max);
        need = std::max(need, (size_t)choose_ptiles(v->device, chunks, ne_max) * K);
    }
    pf_status st = grow_partials(v, need);
    if (st != PF_OK) return st;
    if (w.pix_cap < max_pixels) {
        PF_CUDA(cudaDeviceSynchronize());
        cudaFree(w.points);
        cudaFree(w.block_counts);
        w.points = nullptr;
        w.block_counts = nullptr;
        w.pix_cap = 0;
        PF_CUDA(cudaMalloc(&w.points, sizeof(float4) * (size_t)max_pixels));
        PF_CUDA(cudaMalloc(&w.block_counts, sizeof(int) * ((size_t)max_pixels / BP_CHUNK + 2)));
        w.pix_cap = max_pixels;
    }
    if (!w.state) {
        PF_CUDA(cudaMalloc(&w.state, sizeof(SearchState)));
        PF_CUDA(cudaMalloc(&w.n_points, sizeof(int)));
        PF_CUDA(cudaMalloc(&w.pose_in, 16 * sizeof(double)));
        PF_CUDA(cudaMalloc(&w.pose_out, 16 * sizeof(double)));
        PF_CUDA(cudaMalloc(&w.stats, sizeof(pf_track_stats)));
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
    const int blocks = (int)((npix + BP_CHUNK - 1) / BP_CHUNK);
    PF_CUDA(cudaMallocAsync(&counts, sizeof(int) * blocks, (cudaStream_t)stream));
    st = enqueue_backproject(depth_dev, intr, reinterpret_cast<float4*>(points_dev), counts, n_dev,
                             (cudaStream_t)stream);
    cudaFreeAsync(counts, (cudaStream_t)stream);
    return st;
}

pf_status pf_fitness(const pf_volume* cv, const float* points_dev, int n, const float* poses_dev, int k,
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
    launch_fitness<SRC_POSES>(a, v->fitness_variant, v->cells != nullptr, chunks, s);
    pf::timing_end(pf::KC_FITNESS, s);
    PF_LAUNCHED();
    return PF_OK;
}

pf_status pf_track_reserve(pf_volume* v, int max_pixels, int k_max)
{
    return pf::workspace_reserve(v, max_pixels, k_max);
}

pf_status pf_track_frame_async(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr,
                               const pf_track_params* p, const double* init_pose_dev, double* out_pose_dev,
                               pf_track_stats* stats_dev, void* stream)
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
    st = enqueue_backproject(depth_dev, intr, w.points, w.block_counts, w.n_points, s);
    if (st != PF_OK) return st;

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
        a.stride = stride;
        a.iter = it;
        a.n_ptiles = choose_ptiles(v->device, chunks, ne_max);
        if ((size_t)a.n_ptiles * K > (size_t)w.part_cap) return PF_ERR_INVALID_ARG;
        pf::timing_begin(pf::KC_FITNESS, s);
        launch_fitness<SRC_SEARCH>(a, v->fitness_variant, v->cells != nullptr, chunks, s);
        pf::timing_end(pf::KC_FITNESS, s);
        if (p->update_mode == 0) {
            FitArgs e = a;
            e.K = 1;
            e.n_ptiles = choose_ptiles(v->device, 1, ne_max);
            pf::timing_begin(pf::KC_FITNESS1, s);
            launch_fitness<SRC_EVAL>(e, v->fitness_variant, v->cells != nullptr, 1, s);
            pf::timing_end(pf::KC_FITNESS1, s);
        }
    }
    track_end_kernel<<<1, 32, 0, s>>>(state, w.n_points, out_pose_dev, stats);
    pf::count_launch();
    PF_LAUNCHED();
    return PF_OK;
}

pf_status pf_track_frame(pf_volume* v, const float* depth_dev, const pf_intrinsics* intr, const pf_track_params* p,
                         const double init_pose[16], double out_pose[16], pf_track_stats* stats_host,
                         void* stream)
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
