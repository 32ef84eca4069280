// Ray casting of the fused TSDF (views of the reconstruction and tests).
//
// One thread per pixel marches camera depths z_i = depth_min + i * tau/2 up
// to depth_max through the trilinear field of observed cells (+-1 nodes
// included, unlike the fitness, which needs nodes inside the band); the
// first step from a positive to a non-positive value is refined by linear
// interpolation.  The normal is the normalised central difference of the
// field at +-voxel/2 along each world axis.
#include "pf_internal.cuh"

namespace {

struct RayArgs {
    const void* tsdf;
    const void* weight;
    int nx, ny, nz;
    float inv_vs;
    float org[3];
    float half_vs;
    CamK cam;
    float R[9], t[3];
    float step;
    int nsteps;
    float* depth;
    float* normal;
};

// Trilinear value of an observed cell at world point q; false when the cell
// is outside the grid or has an unobserved node.
template <typename TS>
__device__ inline bool sample_observed(const RayArgs& a, float qx, float qy, float qz, float& out)
{
    const float gx = (qx - a.org[0]) * a.inv_vs;
    const float gy = (qy - a.org[1]) * a.inv_vs;
    const float gz = (qz - a.org[2]) * a.inv_vs;
    if (!(gx >= 0.0f && gx < (float)(a.nx - 1) && gy >= 0.0f && gy < (float)(a.ny - 1) && gz >= 0.0f &&
          gz < (float)(a.nz - 1)))
        return false;
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const int nxy = a.nx * a.ny;
    const int base = (int)fx0 + a.nx * (int)fy0 + nxy * (int)fz0;
    const int off[8] = {0, 1, a.nx, a.nx + 1, nxy, nxy + 1, nxy + a.nx, nxy + a.nx + 1};
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float e = pf_to_float(static_cast<const TS*>(a.tsdf)[base + off[q]]);
        if (e != e) return false;  // unobserved
        v[q] = pf_decode(e);
    }
    const float fx = gx - fx0, fy = gy - fy0, fz = gz - fz0;
    const float x00 = fmaf(fx, v[1] - v[0], v[0]);
    const float x10 = fmaf(fx, v[3] - v[2], v[2]);
    const float x01 = fmaf(fx, v[5] - v[4], v[4]);
    const float x11 = fmaf(fx, v[7] - v[6], v[6]);
    const float y0 = fmaf(fy, x10 - x00, x00);
    const float y1 = fmaf(fy, x11 - x01, x01);
    out = fmaf(fz, y1 - y0, y0);
    return true;
}

template <typename TS>
__global__ void raycast_kernel(RayArgs a)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= a.cam.width || v >= a.cam.height) return;
    const float dcx = __fdiv_rn((float)u - a.cam.cx, a.cam.fx);
    const float dcy = __fdiv_rn((float)v - a.cam.cy, a.cam.fy);
    const float dx = a.R[0] * dcx + a.R[1] * dcy + a.R[2];
    const float dy = a.R[3] * dcx + a.R[4] * dcy + a.R[5];
    const float dz = a.R[6] * dcx + a.R[7] * dcy + a.R[8];
    float hit = 0.0f;
    bool have_prev = false;
    float prev = 0.0f;
    for (int i = 0; i <= a.nsteps; ++i) {
        const float z = fmaf((float)i, a.step, a.cam.dmin);
        float t;
        if (!sample_observed<TS>(a, fmaf(z, dx, a.t[0]), fmaf(z, dy, a.t[1]), fmaf(z, dz, a.t[2]), t)) {
            have_prev = false;
            continue;
        }
        if (have_prev && prev > 0.0f && t <= 0.0f) {
            hit = (z - a.step) + a.step * __fdiv_rn(prev, prev - t);
            break;
        }
        prev = t;
        have_prev = true;
    }
    const size_t pix = (size_t)v * a.cam.width + u;
    a.depth[pix] = hit;
    if (a.normal) {
        float n[3] = {NAN, NAN, NAN};
        if (hit > 0.0f) {
            const float q[3] = {fmaf(hit, dx, a.t[0]), fmaf(hit, dy, a.t[1]), fmaf(hit, dz, a.t[2])};
            float g[3];
            bool ok = true;
            for (int ax = 0; ax < 3 && ok; ++ax) {
                float qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
                qp[ax] += a.half_vs;
                qm[ax] -= a.half_vs;
                float tp, tm;
                ok = sample_observed<TS>(a, qp[0], qp[1], qp[2], tp) && sample_observed<TS>(a, qm[0], qm[1], qm[2], tm);
                g[ax] = tp - tm;
            }
            if (ok) {
                const float len = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                if (len > 0.0f)
                    for (int ax = 0; ax < 3; ++ax) n[ax] = g[ax] / len;
            }
        }
        for (int ax = 0; ax < 3; ++ax) a.normal[3 * pix + ax] = n[ax];
    }
}

}  // namespace

static pf_status pf_raycast_impl(const pf_volume* v, const pf_intrinsics* intr, const double P[16], float* depth_out,
                                 float* normal_out, void* stream)
{
    if (!v || !P || !depth_out) return PF_ERR_INVALID_ARG;
    pf_status st = pf::check_intrinsics(intr);
    if (st != PF_OK) return st;
    for (int q = 0; q < 12; ++q)
        if (!std::isfinite(P[q])) return PF_ERR_INVALID_ARG;
    RayArgs a;
    a.tsdf = v->tsdf;
    a.weight = v->weight;
    a.nx = v->desc.nx;
    a.ny = v->desc.ny;
    a.nz = v->desc.nz;
    a.inv_vs = 1.0f / v->desc.voxel_size;
    a.half_vs = 0.5f * v->desc.voxel_size;
    for (int q = 0; q < 3; ++q) a.org[q] = v->desc.origin[q];
    a.cam = make_cam(intr);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) a.R[3 * r + c] = (float)P[4 * r + c];
        a.t[r] = (float)P[4 * r + 3];
    }
    a.step = 0.5f * v->desc.trunc;
    a.nsteps = (int)floor(((double)intr->depth_max - (double)intr->depth_min) / (double)a.step);
    a.depth = depth_out;
    a.normal = normal_out;
    dim3 block(16, 8);
    dim3 grid((intr->width + 15) / 16, (intr->height + 7) / 8);
    cudaStream_t s = (cudaStream_t)stream;
    pf::timing_begin(pf::KC_RAYCAST, s);
    if (v->desc.tsdf_dtype == PF_F16)
        raycast_kernel<__half><<<grid, block, 0, s>>>(a);
    else if (v->desc.tsdf_dtype == PF_BF16)
        raycast_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(a);
    else if (v->desc.tsdf_dtype == PF_FP8E4M3)
        raycast_kernel<__nv_fp8_e4m3><<<grid, block, 0, s>>>(a);
    else
        raycast_kernel<float><<<grid, block, 0, s>>>(a);
    pf::count_launch();
    pf::timing_end(pf::KC_RAYCAST, s);
    PF_LAUNCHED();
    return PF_OK;
}

// Every entry point that takes a volume keeps its last failing status
// there (pf_volume_last_error).
extern "C" {

pf_status pf_raycast(const pf_volume* v, const pf_intrinsics* intr, const double P[16], float* depth_out,
                     float* normal_out, void* stream)
{
    return pf::keep_status(v, pf_raycast_impl(v, intr, P, depth_out, normal_out, stream));
}

}  // extern "C"
