// Alignment loss, its derivatives and the Gauss-Newton polish.
//
// The residual of a point x under pose T is the TSDF of Sec. III-B at the
// transformed point, r = tsdf(T x) (normalised by tau, trilinear, defined
// when the point falls in a valid cell -- all eight nodes observed and
// inside the band).  The loss of a frame is L = sum r^2.  A pose is
// perturbed on the left, q = Exp(omega) (R x + t) + v with xi = (omega, v),
// so dq/dv = I and dq/domega = -[q - v]x J_l(omega) (J_l the left Jacobian
// of SO(3)); with grad r the gradient of the trilinear interpolant in
// metres,
//     dL/dv = sum 2 r grad r,      dL/domega = J_l^T sum 2 r ((q - v) x grad r),
// and the derivative with respect to the stored value of node n is
// dL/dV_n = sum 2 r w_n(q) over the samples whose cell has node n.
//
// GPU design
//   * align_kernel: grid = (point tiles) x frames.  Per-sample arithmetic is
//     float: each frame's pose is prepared once in FP64 (perturbation,
//     rotation in grid units split into a float pair, translation split into
//     an integer cell and a fraction), and each point's grid coordinate is
//     formed with error-free products and sums, so the cell and fractions
//     carry no rounding at the scale of the grid coordinate.  Node values are
//     read in their storage type.  Per-thread float sums, then FP64 from the
//     block sums on: per-block sums in a fixed order into per-tile partials;
//     align_finish reduces the tiles of each frame in a fixed order and
//     applies J_l^T.  dL/dV goes to an int64 fixed-point
//     accumulator (2^-40 units) by integer atomics: integer addition is
//     associative, so the result does not depend on the order of arrival
//     and the output is bit-reproducible.
//   * Polish: a damped Gauss-Newton (Levenberg-Marquardt) with its state in
//     device memory.  gn_kernel accumulates H = sum J^T J (upper triangle),
//     b = sum J^T r, sum r^2 and the count for the state's candidate pose
//     (float per thread, FP64 across threads and tiles); gn_step (one thread) reduces the tiles, accepts the candidate if
//     it lowers the mean squared residual (lambda /= 10) or drops it
//     (lambda *= 10), solves (H + lambda diag H) d = -b and forms the next
//     candidate [Exp(d_omega) | d_v] T.  No host round trip: a polish is a
//     fixed launch sequence.
#include <algorithm>
#include <climits>
#include <mutex>
#include <unordered_map>

#include "pf_internal.cuh"

namespace {

constexpr int AL_THREADS = 256;
constexpr int AL_TILES = 296;          // most point tiles per frame (2 per SM)
constexpr int AL_BLOCKS = 2432;        // target blocks per launch (2 waves of 8 per SM)
constexpr int RED_THREADS = 256;       // tile reductions
// dL/dV accumulates in int64 units of 2^-40 (fix40 / fixed40_to_float)
constexpr float kRound = 12582912.0f;  // 1.5 * 2^23: adding it rounds |v| < 2^22 to an integer
constexpr int kRoundBits = 0x4B400000;  // its bit pattern
constexpr int GN_VALS = 29;            // 21 (upper H) + 6 (b) + loss + count

struct AlignScratch {
    double* part = nullptr;       // align partials: frames x tiles x 8 (tiles <= AL_TILES)
    size_t part_cap = 0;          // doubles
    long long* acc = nullptr;     // n_nodes fixed-point dL/dV
    double* gn_part = nullptr;    // AL_TILES x GN_VALS
    double* gn_state = nullptr;   // see GnState
    void* frame_pose = nullptr;   // frames x FramePose (the poses prepared once per frame)
    int frame_cap = 0;            // frames
    void* gn_pose = nullptr;      // one PoseF: the polish's candidate, prepared once per step
};

std::mutex g_mu;
std::unordered_map<const pf_volume*, AlignScratch> g_scratch;

struct GnState {
    double T[12];      // current (accepted) pose
    double Tc[12];     // candidate pose
    double H[36], b[6];
    double obj;        // mean squared residual at T
    double lambda;
    int have_cand;     // a candidate is pending evaluation
    int accepted;
    int step;
    int pad;
};

// ---------------------------------------------------------------------------
// FP64 helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline void so3_exp(const double w[3], double R[9])
{
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = sqrt(th2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double kk = 0.0;
            for (int m = 0; m < 3; ++m) kk += K[3 * r + m] * K[3 * m + c];
            R[3 * r + c] = (r == c ? 1.0 : 0.0) + a * K[3 * r + c] + b * kk;
        }
}

// left Jacobian of SO(3): I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2
__device__ inline void so3_left_jacobian(const double w[3], double J[9])
{
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = sqrt(th2);
    double a, b;
    if (th < 1e-6) {
        a = 0.5 - th2 / 24.0;
        b = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = (1.0 - cos(th)) / th2;
        b = (th - sin(th)) / (th2 * th);
    }
    const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double kk = 0.0;
            for (int m = 0; m < 3; ++m) kk += K[3 * r + m] * K[3 * m + c];
            J[3 * r + c] = (r == c ? 1.0 : 0.0) + a * K[3 * r + c] + b * kk;
        }
}

// [Exp(omega) R | Exp(omega) t + v] from a row-major 3x4 (or 4x4) pose
__device__ inline void perturb(const double* P, const double xi[6], double out[12])
{
    double dR[9];
    so3_exp(xi, dR);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += dR[3 * r + m] * P[4 * m + c];
            out[4 * r + c] = acc;
        }
        out[4 * r + 3] += xi[3 + r];
    }
}

struct GridInfo {
    int nx, ny, nz;
    double inv_vs, org[3];
};

// A pose prepared for float sampling: the rotation in grid units as a float
// pair (hi + lo), the translation in grid units as an integer cell o and a
// float fraction b, and the pose in metres as floats (for q itself).
struct PoseF {
    float Ahi[9], Alo[9];
    int o[3];
    float b[3];
    float R[9], t[3];
    int ok;  // the camera lies within 2^21 voxels of the grid
};

__device__ inline void make_posef(const double T[12], const GridInfo& g, PoseF& P)
{
    P.ok = 1;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            const double A = T[4 * r + c] * g.inv_vs;
            P.Ahi[3 * r + c] = (float)A;
            P.Alo[3 * r + c] = (float)(A - (double)P.Ahi[3 * r + c]);
            P.R[3 * r + c] = (float)T[4 * r + c];
        }
        const double tg = (T[4 * r + 3] - g.org[r]) * g.inv_vs;
        if (!(fabs(tg) < 2097152.0)) P.ok = 0;
        const double o = P.ok ? floor(tg) : 0.0;
        P.o[r] = (int)o;
        P.b[r] = (float)(tg - o);
        P.t[r] = (float)T[4 * r + 3];
    }
}

// One frame of pf_align_loss, prepared once per frame (FP64 work that every
// block of the frame would otherwise repeat): the perturbed pose for
// sampling, the translation part v of the perturbation (q - v enters the
// rotation gradient) and the weight 2 W of the node gradient.
struct FramePose {
    PoseF P;
    float V[3];
    float w2;
};

// Copy a record of 4-byte words from global to shared memory with the
// whole block (call from every thread; a barrier follows).
template <typename T>
__device__ inline void block_copy_words(const T* src, T* dst)
{
    static_assert(sizeof(T) % 4 == 0, "4-byte words");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// y = (hi + lo) . x as an integer part and a float fraction, to ~1e-12 of
// |y|: the products are split exactly (p = hi*x rounded, fma(hi, x, -p) its
// error), the three-term sum carries its rounding errors (two-sum), and the
// lo part is added to the error term.  Explicit round-to-nearest intrinsics
// keep the compiler from fusing any step.  False when |y| >= 2^22.
__device__ inline bool row_split(const float* hi, const float* lo, float x, float y, float z, int& yi, float& yf)
{
    const float p0 = __fmul_rn(hi[0], x), p1 = __fmul_rn(hi[1], y), p2 = __fmul_rn(hi[2], z);
    float err = __fadd_rn(__fadd_rn(fmaf(hi[0], x, -p0), fmaf(hi[1], y, -p1)), fmaf(hi[2], z, -p2));
    const float s1 = __fadd_rn(p0, p1);
    float bb = __fsub_rn(s1, p0);
    err = __fadd_rn(err, __fadd_rn(__fsub_rn(p0, __fsub_rn(s1, bb)), __fsub_rn(p1, bb)));
    const float s2 = __fadd_rn(s1, p2);
    bb = __fsub_rn(s2, s1);
    err = __fadd_rn(err, __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, bb)), __fsub_rn(p2, bb)));
    err = fmaf(lo[0], x, fmaf(lo[1], y, fmaf(lo[2], z, err)));
    if (!(fabsf(s2) < 4194304.0f)) return false;
    // nearest integer (ties to even) by adding 1.5 * 2^23, whose unit in the
    // last place is 1; its bits give the integer without a conversion
    const float m = __fadd_rn(s2, kRound);
    const float r = __fsub_rn(m, kRound);
    yi = __float_as_int(m) - kRoundBits;
    yf = __fadd_rn(__fsub_rn(s2, r), err);
    return true;
}

// Trilinear value t, its gradient in grid units, the cell (linear index of
// its lower corner) and the fractions of point x under pose P; false when
// the sample lies in no valid cell (outside the grid, or a node that is
// unobserved or outside the band -- non-finite in the encoded storage).
template <typename TS>
__device__ inline bool sample_f(const TS* tsdf, const GridInfo& g, const PoseF& P, float x, float y, float z,
                                float& t, float dg[3], long long& base, float f[3])
{
    if (!P.ok || !isfinite(x) || !isfinite(y) || !isfinite(z)) return false;
    const int n[3] = {g.nx, g.ny, g.nz};
    long long ci[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        int yi;
        float yf;
        if (!row_split(P.Ahi + 3 * r, P.Alo + 3 * r, x, y, z, yi, yf)) return false;
        const float u = __fadd_rn(yf, P.b[r]);
        // floor(u) the same way with round-down (|u| is a few units)
        const float m = __fadd_rd(u, kRound);
        const float fl = __fsub_rn(m, kRound);
        ci[r] = (long long)P.o[r] + yi + (long long)(__float_as_int(m) - kRoundBits);
        f[r] = __fsub_rn(u, fl);
        if (ci[r] < 0 || ci[r] > n[r] - 2) return false;
    }
    const long long nx = g.nx, nxy = (long long)g.nx * g.ny;
    base = ci[0] + nx * ci[1] + nxy * ci[2];
    const long long off[8] = {0, 1, nx, nx + 1, nxy, nxy + 1, nxy + nx, nxy + nx + 1};
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        v[c] = pf_to_float(tsdf[base + off[c]]);
        if (!isfinite(v[c])) return false;
    }
    const float x00 = fmaf(f[0], v[1] - v[0], v[0]);
    const float x10 = fmaf(f[0], v[3] - v[2], v[2]);
    const float x01 = fmaf(f[0], v[5] - v[4], v[4]);
    const float x11 = fmaf(f[0], v[7] - v[6], v[6]);
    const float y0 = fmaf(f[1], x10 - x00, x00);
    const float y1 = fmaf(f[1], x11 - x01, x01);
    t = fmaf(f[2], y1 - y0, y0);
    const float dx00 = v[1] - v[0], dx10 = v[3] - v[2], dx01 = v[5] - v[4], dx11 = v[7] - v[6];
    const float dy0 = fmaf(f[1], dx10 - dx00, dx00), dy1 = fmaf(f[1], dx11 - dx01, dx01);
    dg[0] = fmaf(f[2], dy1 - dy0, dy0);
    dg[1] = fmaf(f[2], (x11 - x01) - (x10 - x00), x10 - x00);
    dg[2] = y1 - y0;
    return true;
}

__device__ inline void transform_f(const PoseF& P, float x, float y, float z, float q[3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r) q[r] = fmaf(P.R[3 * r], x, fmaf(P.R[3 * r + 1], y, fmaf(P.R[3 * r + 2], z, P.t[r])));
}

// round(x * 2^40) to nearest (ties to even) as an int64, from the bits of
// the float: exactly the value an FP64 multiply by 2^40 and conversion would
// give (both are exact up to that one rounding), without the FP64 pipe.
// Magnitudes of 2^23 and more saturate.
__device__ __forceinline__ long long fix40(float x)
{
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0) return 0;  // zero or subnormal: below 2^-126, rounds to 0
    const int sh = e - 110;  // x * 2^40 = m * 2^(e - 127 - 23 + 40)
    long long r;
    if (sh > 39) {  // |x| >= 2^23: beyond int64
        r = LLONG_MAX;
    } else if (sh >= 0) {
        r = (long long)(((unsigned long long)((b & 0x7fffffu) | 0x800000u)) << sh);
    } else if (sh > -26) {
        const unsigned long long m = (b & 0x7fffffu) | 0x800000u;
        const int s = -sh;
        unsigned long long q = m >> s;
        const unsigned long long rem = m & ((1ull << s) - 1ull), half = 1ull << (s - 1);
        q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
        r = (long long)q;
    } else {
        r = 0;  // below 2^-41
    }
    return (b >> 31) ? -r : r;
}

// Points [beg, end) of this block: n split into gridDim.x contiguous ranges
// of n / G or n / G + 1 points, with 32-bit arithmetic (a 64-bit division
// would run through the FP64 pipe).
__device__ __forceinline__ void block_range(int n, long long& beg, long long& end)
{
    const unsigned G = gridDim.x, b = blockIdx.x, un = (unsigned)n;
    const unsigned q = un / G, r = un % G;
    beg = (long long)b * q + (b < r ? b : r);
    end = beg + q + (b < r ? 1 : 0);
}

// Warps' partial sums (shared sh[warp * NV + i]) to block totals out[i]:
// thread i adds value i over the warps in order, in FP64.
template <int NV>
__device__ inline void warps_to_block(const double* sh, double* out)
{
    const int tid = threadIdx.x;
    if (tid < NV) {
        double s = 0.0;
        for (int w = 0; w < AL_THREADS / 32; ++w) s += sh[w * NV + tid];
        out[tid] = s;
    }
    __syncthreads();
}

// Fixed-order block sum of NV floats per thread, each lane's value carried
// as an unevaluated float pair (s, c) through the warp's shuffle tree with
// error-free additions (TwoSum), so the warp sum keeps about twice float
// precision without the FP64 pipe; warps are then summed in FP64.
// Block totals in out[0 .. NV) (shared), visible to every thread.
template <int NV>
__device__ inline void block_sum_ff(const float* v, double* sh, double* out)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float sv[NV], cv[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        sv[i] = v[i];
        cv[i] = 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float s2 = __shfl_xor_sync(0xffffffffu, sv[i], o), c2 = __shfl_xor_sync(0xffffffffu, cv[i], o);
            // the same operand order on both lanes of a pair (lower lane's
            // value first), so both hold bit-identical results
            const bool low = (lane & o) == 0;
            const float a = low ? sv[i] : s2, b = low ? s2 : sv[i];
            const float ca = low ? cv[i] : c2, cb = low ? c2 : cv[i];
            const float h = __fadd_rn(a, b);
            const float bb = __fsub_rn(h, a);
            const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(h, bb)), __fsub_rn(b, bb));
            sv[i] = h;
            cv[i] = __fadd_rn(__fadd_rn(ca, cb), err);
        }
    if (lane == 0)
        for (int i = 0; i < NV; ++i) sh[warp * NV + i] = (double)sv[i] + (double)cv[i];
    __syncthreads();
    warps_to_block<NV>(sh, out);
}

// Fixed-order block sum of NV floats per thread: the 32 lanes of a warp in
// float (about one sample per lane in the polish, so float keeps ~1e-6 of
// the sum), the warps and thread 0's totals in FP64 (out[0 .. NV)).
template <int NV>
__device__ inline void block_sum_f(float* v, double* sh, double* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if (lane == 0)
        for (int i = 0; i < NV; ++i) sh[warp * NV + i] = (double)v[i];
    __syncthreads();
    warps_to_block<NV>(sh, out);
}

// ---------------------------------------------------------------------------
// Loss and derivatives of F frames
// ---------------------------------------------------------------------------
struct AlignArgs {
    const void* tsdf;
    GridInfo g;
    const float4* pts;
    const int* counts;
    int n_max;
    const double* poses;  // F x 16
    const double* xi;     // F x 6 or null
    const double* dloss;  // F or null
    double* part;         // F x tiles x 8
    long long* acc;       // n_nodes or null
    const FramePose* fposes;  // F, from align_prep
};

// Thread f prepares frame f: its perturbed pose, v and 2 W.
__global__ void align_prep(const double* poses, const double* xi, const double* dloss, GridInfo g, int F,
                           FramePose* out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    double x[6] = {0, 0, 0, 0, 0, 0};
    if (xi)
        for (int i = 0; i < 6; ++i) x[i] = xi[6 * (size_t)f + i];
    double T[12];
    perturb(poses + 16 * (size_t)f, x, T);
    FramePose fp;
    make_posef(T, g, fp.P);
    for (int i = 0; i < 3; ++i) fp.V[i] = (float)x[3 + i];
    fp.w2 = (float)(2.0 * (dloss ? dloss[f] : 1.0));
    out[f] = fp;
}

template <typename TS>
__global__ void __launch_bounds__(AL_THREADS) align_kernel(AlignArgs a)
{
    __shared__ FramePose sF;
    __shared__ double sh[(AL_THREADS / 32) * 8];
    const int f = blockIdx.y, tid = threadIdx.x;
    block_copy_words(a.fposes + f, &sF);
    const PoseF& sP = sF.P;
    const float* sV = sF.V;
    const int n = a.counts ? min(a.counts[f], a.n_max) : a.n_max;
    long long beg, end;
    block_range(n, beg, end);
    const TS* tsdf = static_cast<const TS*>(a.tsdf);
    const float inv_vs = (float)a.g.inv_vs;
    // dL/dV increments in units of 2^-40: round(2 W t w 2^40), formed in
    // float (exact for W = 1, one float rounding otherwise)
    const float w2 = sF.w2;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // L, C, gw[3], gv[3]
    for (long long e = beg + tid; e < end; e += AL_THREADS) {
        const float4 p = __ldg(a.pts + (size_t)f * a.n_max + e);
        float t, dg[3], fr[3];
        long long base;
        if (!sample_f(tsdf, a.g, sP, p.x, p.y, p.z, t, dg, base, fr)) continue;
        float q[3];
        transform_f(sP, p.x, p.y, p.z, q);
        const float gt[3] = {dg[0] * inv_vs, dg[1] * inv_vs, dg[2] * inv_vs};
        const float rr[3] = {q[0] - sV[0], q[1] - sV[1], q[2] - sV[2]};
        const float t2 = 2.0f * t;
        acc[0] = fmaf(t, t, acc[0]);
        acc[1] += 1.0f;
        acc[2] = fmaf(t2, rr[1] * gt[2] - rr[2] * gt[1], acc[2]);
        acc[3] = fmaf(t2, rr[2] * gt[0] - rr[0] * gt[2], acc[3]);
        acc[4] = fmaf(t2, rr[0] * gt[1] - rr[1] * gt[0], acc[4]);
        acc[5] = fmaf(t2, gt[0], acc[5]);
        acc[6] = fmaf(t2, gt[1], acc[6]);
        acc[7] = fmaf(t2, gt[2], acc[7]);
        if (a.acc) {
            const long long nx = a.g.nx, nxy = (long long)a.g.nx * a.g.ny;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float w = ((c & 1) ? fr[0] : 1.0f - fr[0]) * (((c >> 1) & 1) ? fr[1] : 1.0f - fr[1]) *
                                (((c >> 2) & 1) ? fr[2] : 1.0f - fr[2]);
                const long long idx = base + ((c & 1) ? 1 : 0) + (((c >> 1) & 1) ? nx : 0) + (((c >> 2) & 1) ? nxy : 0);
                const long long inc = fix40(w2 * (t * w));
                if (inc != 0) atomicAdd(reinterpret_cast<unsigned long long*>(a.acc + idx), (unsigned long long)inc);
            }
        }
    }
    __shared__ double tot[8];
    block_sum_ff<8>(acc, sh, tot);
    if (tid < 8) a.part[((size_t)f * gridDim.x + blockIdx.x) * 8 + tid] = tot[tid];
}

// Sums of NV values over `tiles` partial records (record y at part + y *
// NV) by one block: thread (i, j) adds value i over tiles j, j + J, ... in
// order, then thread i adds its J partial sums in order (a fixed order
// whatever the scheduling).  Results in out[0 .. NV) of shared memory.
template <int NV>
__device__ inline void tile_sum(const double* part, int tiles, double* sh, double* out)
{
    constexpr int J = RED_THREADS / NV;
    const int tid = threadIdx.x, i = tid % NV, j = tid / NV;
    if (j < J) {
        double acc = 0.0;
        for (int y = j; y < tiles; y += J) acc += part[(size_t)y * NV + i];
        sh[j * NV + i] = acc;
    }
    __syncthreads();
    if (tid < NV) {
        double acc = 0.0;
        for (int q = 0; q < J; ++q) acc += sh[q * NV + tid];
        out[tid] = acc;
    }
    __syncthreads();
}

// one block per frame
__global__ void __launch_bounds__(RED_THREADS) align_finish(const double* part, int tiles, const double* xi,
                                                            const double* dloss, double* loss, int* count,
                                                            double* grad)
{
    __shared__ double sh[RED_THREADS];
    __shared__ double s[8];
    const int f = blockIdx.x;
    tile_sum<8>(part + (size_t)f * tiles * 8, tiles, sh, s);
    if (threadIdx.x != 0) return;
    loss[f] = s[0];
    if (count) count[f] = (int)s[1];
    if (grad) {
        double w[3] = {0, 0, 0};
        if (xi)
            for (int i = 0; i < 3; ++i) w[i] = xi[6 * (size_t)f + i];
        double J[9];
        so3_left_jacobian(w, J);
        const double sc = dloss ? dloss[f] : 1.0;
        for (int i = 0; i < 3; ++i) {
            grad[6 * (size_t)f + i] = sc * (J[i] * s[2] + J[3 + i] * s[3] + J[6 + i] * s[4]);
            grad[6 * (size_t)f + 3 + i] = sc * s[5 + i];
        }
    }
}

// v * 2^-40 rounded to the nearest float (ties to even), by integer
// operations: the same float as the FP64 conversion and multiply for |v| <
// 2^53, without the FP64 pipe (v * 2^-40 stays inside the normal floats).
__device__ __forceinline__ float fixed40_to_float(long long v)
{
    if (v == 0) return 0.0f;
    const unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int msb = 63 - __clzll((long long)m);
    int e = msb - 40;
    unsigned long long q;
    if (msb <= 23) {
        q = m << (23 - msb);
    } else {
        const int s = msb - 23;
        q = m >> s;
        const unsigned long long rem = m & ((1ull << s) - 1ull), half = 1ull << (s - 1);
        q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
        if (q == (1ull << 24)) {
            q >>= 1;
            ++e;
        }
    }
    return __uint_as_float((v < 0 ? 0x80000000u : 0u) | ((unsigned)(e + 127) << 23) | ((unsigned)q & 0x7fffffu));
}

__global__ void fixed_to_float(const long long* acc, float* out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = fixed40_to_float(acc[i]);
}

// ---------------------------------------------------------------------------
// Gauss-Newton polish
// ---------------------------------------------------------------------------
struct GnArgs {
    const void* tsdf;
    GridInfo g;
    const float4* pts;
    const int* n_dev;
    int n_max;
    GnState* st;
    double* part;      // tiles x GN_VALS
    const PoseF* pc;   // the candidate prepared by gn_begin / gn_step
};

template <typename TS>
__global__ void __launch_bounds__(AL_THREADS) gn_kernel(GnArgs a)
{
    __shared__ PoseF sP;
    __shared__ double sh[(AL_THREADS / 32) * GN_VALS];
    const int tid = threadIdx.x;
    if (!a.st->have_cand) return;  // no candidate this step: gn_step ignores the partials
    block_copy_words(a.pc, &sP);
    const int n = a.n_dev ? min(*a.n_dev, a.n_max) : a.n_max;
    long long beg, end;
    block_range(n, beg, end);
    const TS* tsdf = static_cast<const TS*>(a.tsdf);
    const float inv_vs = (float)a.g.inv_vs;
    float acc[GN_VALS];
#pragma unroll
    for (int i = 0; i < GN_VALS; ++i) acc[i] = 0.0f;
    for (long long e = beg + tid; e < end; e += AL_THREADS) {
        const float4 p = __ldg(a.pts + e);
        float t, dg[3], fr[3];
        long long base;
        if (!sample_f(tsdf, a.g, sP, p.x, p.y, p.z, t, dg, base, fr)) continue;
        float q[3];
        transform_f(sP, p.x, p.y, p.z, q);
        const float gt[3] = {dg[0] * inv_vs, dg[1] * inv_vs, dg[2] * inv_vs};
        const float J[6] = {q[1] * gt[2] - q[2] * gt[1], q[2] * gt[0] - q[0] * gt[2], q[0] * gt[1] - q[1] * gt[0],
                            gt[0], gt[1], gt[2]};
        int m = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = r; c < 6; ++c) {
                acc[m] = fmaf(J[r], J[c], acc[m]);
                ++m;
            }
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[21 + r] = fmaf(J[r], t, acc[21 + r]);
        acc[27] = fmaf(t, t, acc[27]);
        acc[28] += 1.0f;
    }
    __shared__ double tot[GN_VALS];
    block_sum_f<GN_VALS>(acc, sh, tot);
    if (tid < GN_VALS) a.part[(size_t)blockIdx.x * GN_VALS + tid] = tot[tid];
}

// solve the 6x6 system A d = y by Gaussian elimination with partial pivoting
__device__ inline bool solve6(double* A, double* y, double d[6])
{
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        for (int r = col + 1; r < 6; ++r)
            if (fabs(A[6 * r + col]) > fabs(A[6 * piv + col])) piv = r;
        if (!(fabs(A[6 * piv + col]) > 0.0)) return false;
        if (piv != col) {
            for (int c = 0; c < 6; ++c) {
                const double tmp = A[6 * col + c];
                A[6 * col + c] = A[6 * piv + c];
                A[6 * piv + c] = tmp;
            }
            const double tmp = y[col];
            y[col] = y[piv];
            y[piv] = tmp;
        }
        for (int r = col + 1; r < 6; ++r) {
            const double m = A[6 * r + col] / A[6 * col + col];
            for (int c = col; c < 6; ++c) A[6 * r + c] -= m * A[6 * col + c];
            y[r] -= m * y[col];
        }
    }
    for (int r = 5; r >= 0; --r) {
        double acc = y[r];
        for (int c = r + 1; c < 6; ++c) acc -= A[6 * r + c] * d[c];
        d[r] = acc / A[6 * r + r];
    }
    return true;
}

// The input pose becomes the first candidate to evaluate.
__global__ void gn_begin(GnState* st, const double* pose_in, GridInfo g, PoseF* pc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < 12; ++i) st->Tc[i] = pose_in[i];
    make_posef(st->Tc, g, *pc);
    st->lambda = 1e-3;
    st->accepted = 0;
    st->step = 0;
    st->obj = INFINITY;
    st->have_cand = 1;
}

// mode 0: take the evaluated input pose as the current one; mode 1: one
// step (accept or drop the evaluated candidate).  Then form the next
// candidate.
__global__ void __launch_bounds__(RED_THREADS) gn_step(GnState* st, const double* part, int tiles, int mode,
                                                       double* pose_out, double* trace, int* accepted_out,
                                                       GridInfo g, PoseF* pc)
{
    __shared__ double sh[RED_THREADS];
    __shared__ double s[GN_VALS];
    const bool evaluated = st->have_cand != 0;
    if (evaluated) tile_sum<GN_VALS>(part, tiles, sh, s);
    if (threadIdx.x != 0) return;
    if (evaluated) {
        const double objc = s[28] > 0.0 ? s[27] / s[28] : INFINITY;
        if (mode == 0 || objc < st->obj) {
            for (int i = 0; i < 12; ++i) st->T[i] = st->Tc[i];
            int m = 0;
            for (int r = 0; r < 6; ++r)
                for (int c = r; c < 6; ++c) {
                    st->H[6 * r + c] = s[m];
                    st->H[6 * c + r] = s[m];
                    ++m;
                }
            for (int r = 0; r < 6; ++r) st->b[r] = s[21 + r];
            st->obj = objc;
            if (mode == 1) {
                st->lambda /= 10.0;
                st->accepted += 1;
            }
        } else {
            st->lambda *= 10.0;
        }
    }
    if (mode == 1) st->step += 1;
    if (trace) trace[st->step] = st->obj;
    // next candidate
    st->have_cand = 0;
    if (st->obj < INFINITY) {
        double A[36], y[6], d[6];
        for (int i = 0; i < 36; ++i) A[i] = st->H[i];
        for (int r = 0; r < 6; ++r) {
            A[7 * r] += st->lambda * st->H[7 * r];
            y[r] = -st->b[r];
        }
        if (solve6(A, y, d)) {
            perturb(st->T, d, st->Tc);
            make_posef(st->Tc, g, *pc);
            st->have_cand = 1;
        }
    }
    if (pose_out) {
        for (int i = 0; i < 12; ++i) pose_out[i] = st->T[i];
        pose_out[12] = pose_out[13] = pose_out[14] = 0.0;
        pose_out[15] = 1.0;
    }
    if (accepted_out) *accepted_out = st->accepted;
}

GridInfo grid_info(const pf_volume* v)
{
    GridInfo g;
    g.nx = v->desc.nx;
    g.ny = v->desc.ny;
    g.nz = v->desc.nz;
    g.inv_vs = 1.0 / (double)v->desc.voxel_size;
    for (int q = 0; q < 3; ++q) g.org[q] = v->desc.origin[q];
    return g;
}

template <template <typename> class K, typename Args>
void launch_storage(const pf_volume* v, dim3 grid, cudaStream_t s, const Args& a)
{
    switch (v->desc.tsdf_dtype) {
    case PF_F16: K<__half>::run(grid, s, a); break;
    case PF_BF16: K<__nv_bfloat16>::run(grid, s, a); break;
    case PF_FP8E4M3: K<__nv_fp8_e4m3>::run(grid, s, a); break;
    default: K<float>::run(grid, s, a); break;
    }
}

template <typename TS>
struct AlignLaunch {
    static void run(dim3 grid, cudaStream_t s, const AlignArgs& a) { align_kernel<TS><<<grid, AL_THREADS, 0, s>>>(a); }
};

template <typename TS>
struct GnLaunch {
    static void run(dim3 grid, cudaStream_t s, const GnArgs& a) { gn_kernel<TS><<<grid, AL_THREADS, 0, s>>>(a); }
};

AlignScratch& scratch_of(const pf_volume* v)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_scratch[v];
}

}  // namespace

namespace pf {
// Frees the scratch of a volume (called by pf_destroy_volume).
void align_release(const pf_volume* v)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch.find(v);
    if (it == g_scratch.end()) return;
    cudaFree(it->second.part);
    cudaFree(it->second.acc);
    cudaFree(it->second.gn_part);
    cudaFree(it->second.gn_state);
    cudaFree(it->second.frame_pose);
    cudaFree(it->second.gn_pose);
    g_scratch.erase(it);
}
}  // namespace pf

extern "C" {

static pf_status pf_align_loss_impl(const pf_volume* v, const float* points_dev, const int* counts_dev, int n_max,
                                    int n_frames, const double* poses_dev, const double* xi_dev,
                                    const double* dloss_dev, double* loss_dev, int* count_dev, double* grad_xi_dev,
                                    float* grad_tsdf_dev, void* stream)
{
    if (!v || !poses_dev || !loss_dev || n_frames < 1 || n_max < 0 || n_frames > 65535) return PF_ERR_INVALID_ARG;
    if (n_max > 0 && !points_dev) return PF_ERR_INVALID_ARG;
    if (((uintptr_t)points_dev & 15) != 0) return PF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    AlignScratch& sc = scratch_of(v);
    const int tiles = std::max(1, std::min(AL_TILES, (AL_BLOCKS + n_frames - 1) / n_frames));
    const size_t need = (size_t)n_frames * tiles * 8;
    if (sc.part_cap < need) {
        cudaFree(sc.part);
        sc.part = nullptr;
        sc.part_cap = 0;
        PF_CUDA(pf::dev_malloc(&sc.part, need * sizeof(double)));
        sc.part_cap = need;
    }
    if (sc.frame_cap < n_frames) {
        cudaFree(sc.frame_pose);
        sc.frame_pose = nullptr;
        sc.frame_cap = 0;
        PF_CUDA(pf::dev_malloc(&sc.frame_pose, (size_t)n_frames * sizeof(FramePose)));
        sc.frame_cap = n_frames;
    }
    if (grad_tsdf_dev && !sc.acc) PF_CUDA(pf::dev_malloc(&sc.acc, v->n_nodes * sizeof(long long)));
    if (grad_tsdf_dev) PF_CUDA(cudaMemsetAsync(sc.acc, 0, v->n_nodes * sizeof(long long), s));
    AlignArgs a;
    a.tsdf = v->tsdf;
    a.g = grid_info(v);
    a.pts = reinterpret_cast<const float4*>(points_dev);
    a.counts = counts_dev;
    a.n_max = n_max;
    a.poses = poses_dev;
    a.xi = xi_dev;
    a.dloss = dloss_dev;
    a.part = sc.part;
    a.acc = grad_tsdf_dev ? sc.acc : nullptr;
    a.fposes = static_cast<const FramePose*>(sc.frame_pose);
    align_prep<<<(n_frames + 63) / 64, 64, 0, s>>>(poses_dev, xi_dev, dloss_dev, a.g, n_frames,
                                                   static_cast<FramePose*>(sc.frame_pose));
    launch_storage<AlignLaunch>(v, dim3(tiles, n_frames), s, a);
    pf::count_launch(2);
    PF_LAUNCHED();
    align_finish<<<n_frames, RED_THREADS, 0, s>>>(sc.part, tiles, xi_dev, dloss_dev, loss_dev, count_dev,
                                                  grad_xi_dev);
    pf::count_launch();
    PF_LAUNCHED();
    if (grad_tsdf_dev) {
        fixed_to_float<<<4 * 152, 256, 0, s>>>(sc.acc, grad_tsdf_dev, v->n_nodes);
        pf::count_launch();
        PF_LAUNCHED();
    }
    return PF_OK;
}

static pf_status pf_polish_impl(const pf_volume* v, const float* points_dev, const int* n_dev, int n_max,
                                double* pose_dev, int steps, double* trace_dev, int* accepted_dev, void* stream)
{
    if (!v || !pose_dev || n_max < 0 || steps < 0 || steps > 1000) return PF_ERR_INVALID_ARG;
    if (n_max > 0 && !points_dev) return PF_ERR_INVALID_ARG;
    if (((uintptr_t)points_dev & 15) != 0) return PF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    AlignScratch& sc = scratch_of(v);
    if (!sc.gn_part) PF_CUDA(pf::dev_malloc(&sc.gn_part, (size_t)AL_TILES * GN_VALS * sizeof(double)));
    if (!sc.gn_state) PF_CUDA(pf::dev_malloc(&sc.gn_state, sizeof(GnState)));
    if (!sc.gn_pose) PF_CUDA(pf::dev_malloc(&sc.gn_pose, sizeof(PoseF)));
    PoseF* pc = static_cast<PoseF*>(sc.gn_pose);
    GnState* st = reinterpret_cast<GnState*>(sc.gn_state);

    GnArgs a;
    a.tsdf = v->tsdf;
    a.g = grid_info(v);
    a.pts = reinterpret_cast<const float4*>(points_dev);
    a.n_dev = n_dev;
    a.n_max = n_max;
    a.st = st;
    a.part = sc.gn_part;
    a.pc = pc;
    // evaluate the input pose, then `steps` candidates
    gn_begin<<<1, 1, 0, s>>>(st, pose_dev, a.g, pc);
    launch_storage<GnLaunch>(v, dim3(AL_TILES), s, a);
    gn_step<<<1, RED_THREADS, 0, s>>>(st, sc.gn_part, AL_TILES, 0, steps == 0 ? pose_dev : nullptr, trace_dev,
                                      accepted_dev, a.g, pc);
    pf::count_launch(3);
    PF_LAUNCHED();
    for (int k = 0; k < steps; ++k) {
        launch_storage<GnLaunch>(v, dim3(AL_TILES), s, a);
        gn_step<<<1, RED_THREADS, 0, s>>>(st, sc.gn_part, AL_TILES, 1, k == steps - 1 ? pose_dev : nullptr,
                                          trace_dev, accepted_dev, a.g, pc);
        pf::count_launch(2);
        PF_LAUNCHED();
    }
    return PF_OK;
}

}  // extern "C"

// Every entry point that takes a volume keeps its last failing status
// there (pf_volume_last_error).
extern "C" {

pf_status pf_align_loss(const pf_volume* v, const float* points_dev, const int* counts_dev, int n_max, int n_frames,
                        const double* poses_dev, const double* xi_dev, const double* dloss_dev, double* loss_dev,
                        int* count_dev, double* grad_xi_dev, float* grad_tsdf_dev, void* stream)
{
    return pf::keep_status(v, pf_align_loss_impl(v, points_dev, counts_dev, n_max, n_frames, poses_dev, xi_dev,
                                                 dloss_dev, loss_dev, count_dev, grad_xi_dev, grad_tsdf_dev, stream));
}

pf_status pf_polish(const pf_volume* v, const float* points_dev, const int* n_dev, int n_max, double* pose_dev,
                    int steps, double* trace_dev, int* accepted_dev, void* stream)
{
    return pf::keep_status(v, pf_polish_impl(v, points_dev, n_dev, n_max, pose_dev, steps, trace_dev, accepted_dev,
                                             stream));
}

}  // extern "C"
