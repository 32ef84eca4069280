/*
 * profusion.h -- C ABI of the GB300 (sm_103a) library for the dense
 * reconstruction back end of PROFusion (arXiv 2509.24236): randomized SE(3)
 * pose search against a TSDF (Sec. III-B) and KinectFusion-style projective
 * TSDF fusion (Sec. III, "Method overview").
 *
 * Conventions used by every call
 *   - Camera frame: x right, y down, z forward.  Pixel (u, v) are integer
 *     indices at pixel centres; depth is the camera z coordinate in metres.
 *     A depth value is usable when finite and in [depth_min, depth_max].
 *   - Poses are camera-to-world, X_w = R X_c + t (Sec. III: P_t = [R_t | t_t]
 *     in the world coordinate system).  4x4 poses are row-major double[16]
 *     (last row 0 0 0 1, not read); fitness poses are row-major float[12]
 *     (the 3x4 block).  Units: metres, radians (search sizes: degrees, cm).
 *   - Volume: nx*ny*nz nodes at origin + voxel_size*(i, j, k), flattened
 *     x-fastest (i + nx*(j + ny*k)).  The TSDF is stored divided by the
 *     truncation tau, so values lie in [-1, 1]; a node with weight 0 is
 *     unobserved.
 *   - Pointers named *_dev are device pointers owned by the caller; *_host
 *     are host pointers owned by the caller.  The library never frees caller
 *     memory.  The library owns the volume's device memory and its workspace
 *     from pf_create_volume until pf_destroy_volume.
 *   - cuda_stream is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream.  All kernels of a call are enqueued on that stream.
 *   - Errors: every call returns pf_status and never aborts.  Arguments are
 *     validated on the host before anything is enqueued (PF_ERR_INVALID_ARG,
 *     nothing enqueued).  A CUDA API failure returns PF_ERR_CUDA; faults of
 *     already-enqueued kernels surface at the next call that synchronises.
 *     Every call that takes a volume also keeps its failing status (any but
 *     PF_OK and PF_ERR_TRACK_LOST) in the volume: pf_volume_last_error.
 *   - Determinism: identical inputs on the same stream give bit-identical
 *     outputs (fixed reduction orders, no floating-point atomics).
 *   - Concurrency: calls that use the same volume must not overlap on
 *     different streams (they share its workspace).
 */
#ifndef PROFUSION_H
#define PROFUSION_H

#if defined(__GNUC__)
#define PF_API __attribute__((visibility("default")))
#else
#define PF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status of every call.  PF_ERR_TIMEOUT is reserved: no call waits on the
 * device (kernels never spin on flags or on one another; ordering comes from
 * stream order). */
typedef enum {
    PF_OK = 0,
    PF_ERR_INVALID_ARG = 1,
    PF_ERR_OOM = 2,
    PF_ERR_CUDA = 3,
    PF_ERR_TIMEOUT = 4,
    PF_ERR_TRACK_LOST = 5,
    PF_ERR_UNSUPPORTED = 6
} pf_status;

/* Pinhole intrinsics of a depth image (Sec. III, "known camera intrinsic
 * parameters").  width, height >= 1; fx, fy > 0; 0 < depth_min <= depth_max. */
typedef struct {
    int width, height;
    float fx, fy, cx, cy;
    float depth_min, depth_max;
} pf_intrinsics;

/* Storage type of the TSDF values (and of the cell view): PF_F32, PF_F16,
 * PF_BF16, or PF_FP8E4M3 -- e4m3 holding the value times 256 (3 mantissa
 * bits; the scale keeps values near the surface out of the e4m3
 * subnormals), with the largest code +-448 standing for the outside-the-band
 * +-1 and the NaN code for unobserved.  Values are rounded to nearest; a
 * value that rounds to +-1 is stored as the outside-the-band code, so the
 * fitness treats such a node as outside the band.  All arithmetic (fusion
 * average, trilinear sample, sums) is float; only the stored values are
 * rounded.  Other codes are rejected with PF_ERR_UNSUPPORTED. */
typedef enum { PF_F32 = 0, PF_F16 = 1, PF_BF16 = 2, PF_FP8E4M3 = 3 } pf_dtype;

/* Dense TSDF grid (Sec. III: "a tensor that records the distance value in
 * each 3D grid").  nx, ny, nz in [2, 4096] with nx*ny*nz < 2^31;
 * voxel_size > 0; trunc (tau, metres) > 0; max_weight in [1, 65535] caps the
 * running-average weight; weight_u8 = 1 stores weights as uint8 (then
 * max_weight <= 255), 0 as float.
 * cell_view: the fitness reads a second copy of the grid in which the eight
 * corner values of every cell are contiguous, kept up to date by fusion.
 * A float grid's records are 32 bytes per node.  The full view of a 16-bit
 * (8-bit) grid keeps a 16-byte (8-byte) record and a 32-byte float record
 * per node; its narrow view keeps the 16-byte (8-byte) record only (lanes
 * on particles then convert on load).  -1 = no view; 1 = the full view;
 * 2 = the narrow view (a float grid takes 1); 0 = automatic: the full
 * view when the whole volume (grid, weights, view) fits in half of the
 * device memory free at creation (decoding narrow records on load slows the
 * search once the particles converge), else the narrow view when that
 * fits, else none.  pf_volume_info reports the choice.
 * search_dtype: storage type of the records in the cell view, which is what
 * the search (pf_track_frame, and pf_fitness with the default layout) reads.
 * PF_F32 (0): the tsdf storage type.  PF_F16, PF_BF16 or PF_FP8E4M3 with a
 * float grid: a narrow search view of the float master grid -- fusion keeps
 * averaging in float, and every refresh of the view rounds the current node
 * values into it once (to nearest; a value that rounds to +-1 becomes the
 * outside-the-band code), so the search samples that rounded grid while
 * fusion accumulates no rounding.  It needs a cell view (cell_view -1 is
 * PF_ERR_INVALID_ARG; automatic takes the full view when it fits, else the
 * narrow one, else fails with PF_ERR_OOM).  Any other combination with a
 * narrower search type is PF_ERR_UNSUPPORTED. */
typedef struct {
    int nx, ny, nz;
    float voxel_size;
    float trunc;
    float origin[3];
    pf_dtype tsdf_dtype;
    int weight_u8;
    int max_weight;
    int cell_view;
    pf_dtype search_dtype;
} pf_volume_desc;

/* Parameters of the randomized optimization (Sec. III-B, defaults Sec. IV-A:
 * n_iters 20, k_sched {1024, 3072, 10240}, decim_sched {8, 16, 32},
 * init 10 deg / 10 cm, beta 0.1).
 *   n_iters        1..PF_MAX_ITERS iterations, no early exit.
 *   k_sched[i%3]   particles of iteration i (1..k_max; particle 0 = current
 *                  pose), decim_sched[i%3] keeps every n-th valid point (>= 1).
 *   templates_dev  k_max x 6 floats (device): row k = (rx, ry, rz, tx, ty, tz),
 *                  the delta pose of particle k in units of the search size;
 *                  row 0 must be zero.  Delta pose = [Exp(omega*pi/180*r) |
 *                  v/100*t].
 *   update_mode    0: pose <- mean of the advantage set {k : E_k < E_0}
 *                  composed onto the pose (the paper's update);
 *                  1: pose <- best particle.
 *   compose_mode   0: dP * P as written (rotation about the world origin);
 *                  1: rotation about the camera centre (R' = dR R, t' = t + dt).
 *   min_valid_frac the frame is lost when particle 0 of the first iteration
 *                  has fewer than this fraction of the evaluated points valid
 *                  (or none). */
typedef struct {
    int n_iters;
    int k_sched[3];
    int decim_sched[3];
    double init_rot_deg, init_trans_cm, beta;
    const float* templates_dev;
    int k_max;
    int update_mode;
    int compose_mode;
    float min_valid_frac;
} pf_track_params;

#define PF_MAX_ITERS 32

/* Per-frame record of the search; entries [0, n_iters) are filled.
 * E values are fitness (mean |tsdf| over valid points, +inf if none). */
typedef struct {
    int n_points;                   /* valid back-projected points (all, before decimation) */
    int n_iters;                    /* iterations run */
    int status;                     /* PF_OK or PF_ERR_TRACK_LOST */
    int reserved;
    float E0[PF_MAX_ITERS];         /* fitness of the pose entering iteration i (particle 0) */
    float E_best[PF_MAX_ITERS];     /* smallest particle fitness */
    float E_new[PF_MAX_ITERS];      /* fitness of the updated pose (search-size update) */
    int best[PF_MAX_ITERS];         /* index of the best particle (lowest among ties) */
    int n_adv[PF_MAX_ITERS];        /* size of the advantage set */
    int n_valid0[PF_MAX_ITERS];     /* valid points of particle 0 */
    int n_eval[PF_MAX_ITERS];       /* points evaluated (after decimation) */
    int k_used[PF_MAX_ITERS];       /* particles evaluated */
    double s[PF_MAX_ITERS][2];      /* search size (deg, cm) used in iteration i */
    double pose[PF_MAX_ITERS][12];  /* pose after iteration i, row-major 3x4 */
} pf_track_stats;

typedef struct pf_volume pf_volume;

/* Allocate a volume on the current device, all nodes unobserved.
 * Errors: INVALID_ARG (bad desc or out == NULL), UNSUPPORTED (dtype/weight
 * storage not provided), OOM, CUDA. */
PF_API pf_status pf_create_volume(const pf_volume_desc* desc, void* cuda_stream, pf_volume** out);

/* Free the volume and its workspace (synchronises the device). NULL is OK. */
PF_API pf_status pf_destroy_volume(pf_volume* vol);

/* The last failing status (not PF_OK, not PF_ERR_TRACK_LOST) returned by a
 * call on this volume, PF_OK if none since creation or the last clear;
 * clear != 0 resets it to PF_OK.  PF_ERR_INVALID_ARG for a NULL volume. */
PF_API pf_status pf_volume_last_error(pf_volume* vol, int clear);

/* Mark every node unobserved (asynchronous on cuda_stream). */
PF_API pf_status pf_reset_volume(pf_volume* vol, void* cuda_stream);

/* Copy a whole grid in from / out to host float arrays of nx*ny*nz values:
 * normalised tsdf and weight (weight 0 = unobserved; download reports tsdf 1
 * there).  Synchronous; intended for tests and checkpoints. */
PF_API pf_status pf_volume_upload(pf_volume* vol, const float* tsdf_host, const float* weight_host);
PF_API pf_status pf_volume_download(const pf_volume* vol, float* tsdf_host, float* weight_host);

/* Fuse one depth image (height x width floats, row-major, device) taken at
 * cam_to_world into the volume (Sec. III fusion, KinectFusion rule): every
 * node with camera depth z_c > 0 projecting to pixel (floor(u+1/2),
 * floor(v+1/2)) inside the image with a usable depth d gets sdf = d - z_c; if
 * sdf >= -tau it is averaged in as t = min(1, sdf/tau) with weight 1:
 * tsdf <- (w tsdf + t)/(w + 1), w <- min(w + 1, max_weight). */
PF_API pf_status pf_integrate(pf_volume* vol, const float* depth_dev, const pf_intrinsics* intr,
                       const double cam_to_world[16], void* cuda_stream);

/* As pf_integrate, with the pose in device memory (double[16]); nothing
 * synchronises, so a frame's search and fusion can run back to back on the
 * device (and be captured in a CUDA graph). */
PF_API pf_status pf_integrate_async(pf_volume* vol, const float* depth_dev, const pf_intrinsics* intr,
                                    const double* cam_to_world_dev, void* cuda_stream);

/* out_dev = a_dev * b_dev for row-major 4x4 double poses in device memory,
 * in FP64: the initial pose of a frame, P_t^(0) = P_{t-1} P_(t,t-1)
 * (Sec. III-A).  out_dev may alias neither input. */
PF_API pf_status pf_pose_compose(const double* a_dev, const double* b_dev, double* out_dev, void* cuda_stream);

/* Back-project a depth image into metric camera-frame points (Sec. III,
 * problem setting): pixel (u, v) with usable depth z gives
 * ((u - cx) z / fx, (v - cy) z / fy, z).  Points of usable pixels are
 * written as float4 (x, y, z, 0) to points_dev (capacity entries,
 * >= width*height) in tile order: the image is cut into 8 x 4-pixel tiles,
 * taken row-major over tiles and row-major inside a tile (so 32 consecutive
 * points are one compact image patch).  The count is written to *n_dev
 * (device int).  No decimation here: the search keeps every n-th point of
 * this order itself. */
PF_API pf_status pf_backproject(const float* depth_dev, const pf_intrinsics* intr, float* points_dev,
                         int capacity, int* n_dev, void* cuda_stream);

/* Fitness of k poses against n points (Sec. III-B):
 * E_k = (1/|X_k|) sum_{x in X_k} |tsdf(T_k x)| with trilinear lookup, where
 * X_k holds the points whose containing cell lies inside the grid with all
 * eight nodes observed and within the truncation (|tsdf| < 1).
 *   points_dev  n x 4 floats (x, y, z, ignored), camera frame.
 *   poses_dev   k x 12 floats, row-major 3x4 camera-to-world.
 *   fitness_dev k floats: E_k (+inf when X_k is empty); count_dev k ints: |X_k|.
 * n >= 0 (n = 0 gives +inf / 0), 1 <= k <= 65536. */
PF_API pf_status pf_fitness(const pf_volume* vol, const float* points_dev, int n, const float* poses_dev,
                     int k, float* fitness_dev, int* count_dev, void* cuda_stream);

/* As pf_fitness, but allocates no device memory (no cudaMalloc, no library
 * allocator), for callers that must not allocate once they are running --
 * e.g. a process whose device memory is owned by another allocator, or a
 * real-time loop that cannot afford the device-wide synchronisation an
 * allocation implies.  The paper has no counterpart: this is an interface
 * variant of pf_fitness, with identical semantics and arguments.
 *   Scratch: the kernel's partial sums live in one fixed array of
 *   PF_NOALLOC_MAX_SLOTS (point tile, pose) slots (about 512 KiB) that every
 *   device which loads the library holds until the process exits.
 *   k > PF_NOALLOC_MAX_SLOTS is rejected with PF_ERR_INVALID_ARG before
 *   anything is enqueued; smaller k may use fewer point tiles than
 *   pf_fitness, which changes only the float summation order.
 *   The volume's device must be the current device (else
 *   PF_ERR_INVALID_ARG: the array used is the current device's).
 *   The first call on a device is its set-up: it looks up the array's
 *   device address and loads the code of every fitness kernel the call can
 *   launch (any storage type, layout or lane mapping), which may allocate;
 *   make that first call before any stream capture.  Later calls on that
 *   device allocate nothing (pf_alloc_count does not move).
 *   All calls share the array: calls that overlap on the GPU (other streams,
 *   other host threads) race and must be serialised by the caller. */
#define PF_NOALLOC_MAX_SLOTS 65536
PF_API pf_status pf_fitness_noalloc(const pf_volume* vol, const float* points_dev, int n, const float* poses_dev,
                                    int k, float* fitness_dev, int* count_dev, void* cuda_stream);

/* Randomized pose optimization of one frame (Sec. III-B): back-projects the
 * depth, then runs params->n_iters iterations of sample / evaluate / select /
 * update, starting from init_pose with search size (init_rot_deg,
 * init_trans_cm).  Pose composition and re-orthonormalisation run in FP64 on
 * the device.  out_pose receives the refined pose, or init_pose when the
 * frame is lost (then PF_ERR_TRACK_LOST is returned).  stats_or_null
 * receives the per-iteration record.  Synchronises cuda_stream.
 * The first call on a volume (or one with a larger frame or k_max) allocates
 * workspace. */
PF_API pf_status pf_track_frame(pf_volume* vol, const float* depth_dev, const pf_intrinsics* intr,
                         const pf_track_params* params, const double init_pose[16], double out_pose[16],
                         pf_track_stats* stats_or_null, void* cuda_stream);

/* As pf_track_frame, but init_pose_dev / out_pose_dev (double[16]) and the
 * optional stats live in device memory and nothing synchronises, so the call
 * can be captured in a CUDA graph once the workspace exists (call
 * pf_track_reserve or one pf_track_frame first).  The lost status is
 * stats->status; out_pose_dev then holds init_pose_dev. */
PF_API pf_status pf_track_frame_async(pf_volume* vol, const float* depth_dev, const pf_intrinsics* intr,
                               const pf_track_params* params, const double* init_pose_dev,
                               double* out_pose_dev, pf_track_stats* stats_dev_or_null,
                               void* cuda_stream);

/* Allocate the tracking workspace for frames up to max_pixels pixels and up
 * to k_max particles (synchronous). */
PF_API pf_status pf_track_reserve(pf_volume* vol, int max_pixels, int k_max);

/* Ray-cast the fused surface seen from cam_to_world: for each pixel, march
 * camera depths z_i = depth_min + i * (trunc/2) up to depth_max through the
 * trilinear field of observed cells; the first step from a positive to a
 * non-positive value is refined by linear interpolation.  depth_out_dev
 * (height x width floats) gets that depth or 0; normal_out_dev_or_null
 * (height x width x 3 floats) gets the unit world-frame gradient there
 * (central differences at +-voxel/2) or NaN. */
PF_API pf_status pf_raycast(const pf_volume* vol, const pf_intrinsics* intr, const double cam_to_world[16],
                     float* depth_out_dev, float* normal_out_dev_or_null, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent sequences (each with its own volume, camera and
 * search parameters; sizes may differ) stepped together.  One step is one
 * frame of every sequence: the initial pose is the sequence's current pose
 * times its relative pose input (P_t^(0) = P_{t-1} P_(t,t-1), Sec. III-A),
 * the randomized optimization of Sec. III-B runs from it, and the frame is
 * fused at the result (Sec. III).  Each search iteration of all sequences is
 * one launch over the thread blocks of every sequence (each sequence keeps
 * its own arguments, partial sums and selection, so its results equal those
 * of pf_track_frame_async with the same point tiling), and with use_graph
 * the whole step is captured once as a CUDA graph and replayed.
 *   vols     n distinct volumes (a volume holds one sequence's search state),
 *            all with the same tsdf storage type and fitness layout (the
 *            plain layout is not supported); their workspaces are reserved
 *            here.  The batch does not own them; destroy it first.
 *   intrs, params  n entries each (templates stay owned by the caller).
 * Buffers owned by the batch, on the device (pf_batch_buffers): per sequence
 * the depth image (width x height float, written by the caller before each
 * step), the relative pose input and the current pose (double[16] each; the
 * current pose starts as the identity -- write the first frame's pose
 * there) and the search record of the last step.
 * pf_batch_fuse fuses every sequence's depth at its current pose (the first
 * frame).  pf_batch_step enqueues one step on cuda_stream (the first step
 * with use_graph captures the graph on a private stream; later steps replay
 * it; nothing synchronises).  pf_batch_autotune tunes two axes of the
 * batched launches by timing the first search iteration of the current
 * frames on copies of the search state: the evaluated points per thread
 * block (at the initial and at a 1e-3 contracted search size), then the
 * lane-mapping threshold -- the reach of a particle chunk, in voxels, below
 * which particles take the lanes of a warp instead of points -- at search
 * sizes 0.3, 0.1 and 0.03 of the initial one, where chunks change mapping
 * (for sequences whose fitness variant leaves the mapping automatic; the
 * mapping changes only the order of the float sums); it synchronises and
 * drops any captured graph.  pf_batch_set_points_per_block (>= 1024) and
 * pf_batch_set_mapping_threshold (voxels; <= 0: each volume's default, 5
 * with a cell view and 12 without) set them directly; pf_batch_tuning
 * reports both (threshold 0 = the defaults).  Errors: PF_ERR_INVALID_ARG for
 * bad arguments (before any allocation), PF_ERR_UNSUPPORTED for mixed
 * storage types or layouts. */
typedef struct pf_batch pf_batch;
PF_API pf_status pf_batch_create(int n, pf_volume* const* vols, const pf_intrinsics* intrs,
                                 const pf_track_params* params, int use_graph, pf_batch** out);
PF_API pf_status pf_batch_destroy(pf_batch* batch);
PF_API pf_status pf_batch_buffers(pf_batch* batch, int i, float** depth_dev, double** rel_pose_dev,
                                  double** pose_dev, pf_track_stats** stats_dev);
PF_API pf_status pf_batch_fuse(pf_batch* batch, void* cuda_stream);
PF_API pf_status pf_batch_step(pf_batch* batch, void* cuda_stream);
PF_API pf_status pf_batch_autotune(pf_batch* batch, void* cuda_stream, int* points_per_block_out);
PF_API pf_status pf_batch_set_points_per_block(pf_batch* batch, int points_per_block);
PF_API pf_status pf_batch_set_mapping_threshold(pf_batch* batch, float voxels);
PF_API pf_status pf_batch_tuning(const pf_batch* batch, int* points_per_block, float* mapping_threshold);

/* Alignment loss of n_frames poses against their frames' points, and its
 * derivatives -- the gradient counterpart of the fitness (Sec. III-B: the
 * residual of a point is the TSDF at the transformed point, normalised by
 * tau and trilinear, defined when the point falls in a valid cell; the loss
 * of a frame is the sum of squared residuals).
 *   points_dev   n_frames x n_max float4 (x, y, z, unused), camera frame,
 *                metres, 16-byte aligned; frame f uses its first
 *                counts_dev[f] rows (counts_dev NULL: all n_max).
 *   poses_dev    n_frames x 16 double, camera-to-world, row-major.
 *   xi_dev       n_frames x 6 double (omega, v) or NULL (zero): frame f is
 *                evaluated at q = Exp(omega) (R x + t) + v (a perturbation on
 *                the left; Exp = Rodrigues).
 *   dloss_dev    n_frames double or NULL (ones): upstream gradient of each
 *                frame's loss, scaling the derivatives below.
 *   loss_dev     out, n_frames double: sum of squared residuals.
 *   count_dev    out, n_frames int or NULL: points in valid cells.
 *   grad_xi_dev  out, n_frames x 6 double or NULL: dloss_f * dL_f / dxi_f
 *                at xi_f (rotation part through the left Jacobian of SO(3)).
 *   grad_tsdf_dev out, n_nodes float or NULL: sum_f dloss_f dL_f/dV, the
 *                derivative with respect to the stored (tau-normalised) node
 *                values at fixed cell validity; accumulated in 2^-40 fixed
 *                point, so it is independent of execution order.
 * Arithmetic: each point's grid coordinate is formed in float with
 * error-free products and sums (no rounding at the scale of the coordinate)
 * and each sample's residual and gradient in float; the per-frame pose
 * preparation and the sums across warps and thread blocks are FP64; dL/dV is
 * accumulated in 2^-40 fixed point (int64).  The first call allocates library scratch
 * (n_frames x 2368 doubles; with grad_tsdf_dev also n_nodes x 8 bytes) kept
 * until the volume is destroyed.  Asynchronous on cuda_stream. */
PF_API pf_status pf_align_loss(const pf_volume* vol, const float* points_dev, const int* counts_dev, int n_max,
                               int n_frames, const double* poses_dev, const double* xi_dev, const double* dloss_dev,
                               double* loss_dev, int* count_dev, double* grad_xi_dev, float* grad_tsdf_dev,
                               void* cuda_stream);

/* Gradient polish of a pose after the search (a refinement of Sec. III-B's
 * result on the same residuals): damped Gauss-Newton (Levenberg-Marquardt)
 * on r_j = tsdf(T x_j) over the points in valid cells, with Jacobian
 * J_j = grad r^T [-[q]x | I] for a left perturbation.  Each step solves
 * (H + lambda diag(H)) d = -b (H = sum J^T J, b = sum J^T r) and tries the
 * candidate [Exp(d_omega) | d_v] T; it is accepted only when it lowers the
 * mean squared residual (then lambda /= 10), otherwise dropped
 * (lambda *= 10); lambda starts at 1e-3.
 *   points_dev   n_max float4 (camera frame, metres), 16-byte aligned; the
 *                first *n_dev rows are used (n_dev NULL: all n_max), e.g.
 *                the output of pf_backproject.
 *   pose_dev     in/out, double[16] on the device.
 *   steps        candidates to try (0..1000).
 *   trace_dev    out, steps + 1 doubles or NULL: the objective before the
 *                first step and after each step.
 *   accepted_dev out, int or NULL: accepted steps.
 * All state stays on the device (no synchronisation; capturable once the
 * scratch exists -- the first call allocates it). */
PF_API pf_status pf_polish(const pf_volume* vol, const float* points_dev, const int* n_dev, int n_max,
                           double* pose_dev, int steps, double* trace_dev, int* accepted_dev, void* cuda_stream);

/* Fitness kernel variant used by pf_fitness and the search of this volume,
 * variant = layout + 4 * mapping (0 is the default everywhere).
 *   layout  0: the cell view when the volume has one, else 2;
 *           1: the plain float form, the performance baseline: every
 *              sample's grid coordinate A x + c in float from the particle's
 *              absolute transform, floor, an explicit range test, eight tsdf
 *              and eight weight loads with all eight nodes tested; lanes on
 *              points only (the mapping is ignored); float storage only;
 *           2: the tsdf array alone, whose encoding makes a cell's validity
 *              a property of its interpolated value;
 *           3: the cell view (PF_ERR_INVALID_ARG if the volume has none).
 *   mapping 0: chosen per block of points from the spread of the particles;
 *           1: neighbouring points on the lanes of a warp;
 *           2: particles on the lanes of a warp.
 * Layouts 2 and 3 evaluate the same samples (bit-identical for a given
 * mapping; mappings differ only by the float summation order).  Layout 1
 * rounds each sample position once at the scale of the grid coordinate
 * (instead of forming it from exact reference products), so its values
 * differ from the others by that rounding. */
PF_API pf_status pf_set_fitness_variant(pf_volume* vol, int variant);

/* Device memory a volume holds for its grid, weights and cell view
 * (workspaces of the search excluded) in *storage_bytes, and the cell view
 * it took in *cell_view (-1 none, 1 full, 2 narrow; see pf_volume_desc).
 * Either pointer may be NULL.  PF_ERR_INVALID_ARG for a NULL volume. */
PF_API pf_status pf_volume_info(const pf_volume* vol, unsigned long long* storage_bytes, int* cell_view);

PF_API const char* pf_status_string(pf_status status);

/* --- instrumentation ---------------------------------------------------- */

/* Number of kernels this library has enqueued since it was loaded. */
PF_API unsigned long long pf_launch_count(void);

/* Number of device allocations (cudaMalloc / cudaMallocAsync) this library
 * has made since it was loaded. */
PF_API unsigned long long pf_alloc_count(void);

/* Memory ceilings for the fitness kernel's roofline (the fitness of Sec.
 * III-B reads one 32-byte cell record per sample, mostly from L2).  Reads
 * loads_per_thread 32-byte records per thread from buf_dev (n_records
 * records of 8 floats, n_records a multiple of 32 in [32, 2^31], 32-byte
 * aligned; size it to fit in L2 and fill it before timing):
 *   mode 0  each warp reads 32 consecutive records (1 KiB) at a random
 *           1 KiB-aligned position, bypassing L1: L2 -> SM bandwidth;
 *   mode 1  each lane reads one record at a random position with the
 *           fitness kernel's 256-bit read-only load: a fully scattered gather.
 * Positions follow h <- 1664525 h + 1013904223 (mod 2^32) per warp (mode 0)
 * or per thread (mode 1), seeded by the murmur3 finaliser of the warp or
 * thread index; record = floor(h * n / 2^32) (mode 0: block * 32 + lane).
 * out_dev gets one float per thread: the sum of the values it loaded (each
 * record's eight values as ((v0+v1)+(v2+v3))+((v4+v5)+(v6+v7)), added in
 * load order).  *threads_out receives the thread count (out_dev NULL:
 * only that, nothing launched).  Bytes read = threads x loads x 32; time it
 * with events on cuda_stream.  Launches one kernel; no synchronisation. */
PF_API pf_status pf_gather_probe(const float* buf_dev, long long n_records, int mode, int loads_per_thread,
                                 float* out_dev, long long* threads_out, void* cuda_stream);

/* When enabled, every launch of the named kernel class ("fitness": the
 * search and pf_fitness launches; "fitness1": the single-pose evaluation of
 * the mean update; "integrate"; "refresh": the cell-view update after
 * fusion; "backproject"; "raycast") is bracketed by
 * CUDA events on its stream.  pf_kernel_timing synchronises those events, returns the summed
 * device time (ms) and launch count since the last query, and clears them. */
PF_API pf_status pf_set_kernel_timing(int enable);
PF_API pf_status pf_kernel_timing(const char* kernel_class, double* total_ms, long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* PROFUSION_H */
