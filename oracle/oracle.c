/*
 * Plain FP64 CPU oracle for the randomized pose search and TSDF fusion of
 * PROFusion (arXiv 2509.24236).  TEST INFRASTRUCTURE ONLY: it exists so that
 * the CUDA library can be checked against an independent, obviously correct
 * restatement of the method.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg call it; the library never does.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Sources followed, step by step:
 *   problem setting (Sec. III, "Problem setting"): depth -> metric points;
 *   fusion "the same as KinectFusion" (Sec. III, "Method overview");
 *   randomized optimization (Sec. III-B): delta poses sampled within the
 *     search size s = (omega deg, v cm), global transform dP_k * P, fitness
 *     E = mean over valid points of |TSDF(dP_k P x)| / tau, advantage set
 *     {k : E_k < E(P)}, mean delta pose, P <- mean * P,
 *     s <- beta s + (1 - beta) E(P) s with beta = 0.1;
 *   defaults (Sec. IV-A): s^(1) = (10 deg, 10 cm), particle counts
 *     1024/3072/10240 and point down-sampling 1/8, 1/16, 1/32 alternating,
 *     at most 20 iterations.
 *   gradient refinement (this project's addition on the residual of Sec.
 *     III-B): the alignment loss sum tsdf(T x)^2, its derivatives with
 *     respect to a left pose perturbation and to the node values, and a
 *     damped Gauss-Newton polish of the pose.
 * Where the paper is silent the readings below are used (each is marked
 * "reading:" at its place): tsdf stored normalised by tau, trilinear lookup,
 * validity = all eight cell nodes observed with |tsdf| < 1, empty set -> E = +inf,
 * decoupled delta pose (Exp(rotation vector), translation), rotation mean =
 * mean of rotation vectors, projective z-distance fusion with weight cap.
 *
 * Everything is double precision except the inputs that arrive as float
 * (depth images, templates, fitness poses), which are promoted exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

typedef struct {
    int width, height;
    double fx, fy, cx, cy, depth_min, depth_max;
} or_intr;

typedef struct {
    int nx, ny, nz;
    double voxel_size, trunc;
    double origin[3];
    int max_weight;
} or_grid;

typedef struct {
    int n_iters;
    int k_sched[3];
    int decim_sched[3];
    double s0_deg, s0_cm, beta;
    int update_mode;   /* 0: advantage-set mean (Sec. III-B), 1: best particle */
    int compose_mode;  /* 0: dP * P literally, 1: rotation about the camera centre */
    double min_valid_frac;
} or_params;

#define OR_MAX_ITERS 32
typedef struct {
    int n_points, n_iters, lost, pad;
    double E0[OR_MAX_ITERS], E_best[OR_MAX_ITERS], E_new[OR_MAX_ITERS];
    int best[OR_MAX_ITERS], n_adv[OR_MAX_ITERS], n_valid0[OR_MAX_ITERS], n_eval[OR_MAX_ITERS];
    int k_used[OR_MAX_ITERS], pad2;
    double s[OR_MAX_ITERS][2];
    double pose[OR_MAX_ITERS][12];
    /* test aids: smallest |E_k - E_0| / E_0 over k != 0 and the relative gap
       between the two smallest E_k, per iteration */
    double adv_margin[OR_MAX_ITERS], best_gap[OR_MAX_ITERS];
} or_stats;

static size_t node_index(const or_grid* g, long i, long j, long k)
{
    return (size_t)i + (size_t)g->nx * ((size_t)j + (size_t)g->ny * (size_t)k);
}

/* ------------------------------------------------------------------------ */
/* Problem setting: each depth pixel back-projects to a metric point.        */
/* ------------------------------------------------------------------------ */

static int depth_valid(float z, const or_intr* in)
{
    /* reading: a measurement is usable when finite and inside the sensor range */
    return isfinite(z) && (double)z >= in->depth_min && (double)z <= in->depth_max;
}

/* Points of the valid pixels; the j-th valid pixel is kept when
 * j mod stride == 0 (down-sampling, Sec. IV-A).  Returns the count.
 * reading: the order of the point cloud (which decides the down-sampled
 * subset) is tile order -- the image cut into 8 x 4-pixel tiles, taken
 * row-major over tiles and row-major inside each tile. */
long or_backproject(const float* depth, const or_intr* in, int stride, double* pts)
{
    long j = 0, n = 0;
    int tiles_x = (in->width + 7) / 8, tiles_y = (in->height + 3) / 4;
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx)
            for (int dv = 0; dv < 4; ++dv)
                for (int du = 0; du < 8; ++du) {
                    int u = tx * 8 + du, v = ty * 4 + dv;
                    if (u >= in->width || v >= in->height) continue;
                    float z = depth[(size_t)v * in->width + u];
                    if (!depth_valid(z, in)) continue;
                    if (j % stride == 0) {
                        double zd = (double)z;
                        pts[3 * n + 0] = ((double)u - in->cx) * zd / in->fx;
                        pts[3 * n + 1] = ((double)v - in->cy) * zd / in->fy;
                        pts[3 * n + 2] = zd;
                        ++n;
                    }
                    ++j;
                }
    return n;
}

/* ------------------------------------------------------------------------ */
/* TSDF lookup: trilinear interpolation on the node lattice.                 */
/* ------------------------------------------------------------------------ */

/* reading: the TSDF at a point is the trilinear interpolation of the eight
 * nodes of the cell containing it, written as successive linear
 * interpolations along x, then y, then z.  The point is usable only when the
 * cell lies inside the grid and all eight nodes are usable: observed
 * (weight > 0) and, when `band` is set, within the truncation distance
 * (|tsdf| < 1) -- the "valid grids" of Sec. III-B.  Returns 1 and the value,
 * or 0.  gcoord (optional) receives the continuous grid coordinates. */
static int sample_cell(const double* tsdf, const double* weight, const or_grid* g,
                       const double q[3], int band, double* val, double gcoord[3])
{
    double gc[3], f[3];
    long i0[3];
    int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        gc[a] = (q[a] - g->origin[a]) / g->voxel_size;
        if (gcoord) gcoord[a] = gc[a];
    }
    for (int a = 0; a < 3; ++a) {
        if (!(gc[a] >= 0.0 && gc[a] < (double)(n[a] - 1))) return 0;
        i0[a] = (long)floor(gc[a]);
        f[a] = gc[a] - (double)i0[a];
    }
    double v[8];
    for (int c = 0; c < 8; ++c) {
        size_t idx = node_index(g, i0[0] + (c & 1), i0[1] + ((c >> 1) & 1), i0[2] + ((c >> 2) & 1));
        if (!(weight[idx] > 0.0)) return 0;
        if (band && !(fabs(tsdf[idx]) < 1.0)) return 0;
        v[c] = tsdf[idx];
    }
    /* corners c = dx + 2 dy + 4 dz */
    double x00 = v[0] + f[0] * (v[1] - v[0]);
    double x10 = v[2] + f[0] * (v[3] - v[2]);
    double x01 = v[4] + f[0] * (v[5] - v[4]);
    double x11 = v[6] + f[0] * (v[7] - v[6]);
    double y0 = x00 + f[1] * (x10 - x00);
    double y1 = x01 + f[1] * (x11 - x01);
    *val = y0 + f[2] * (y1 - y0);
    return 1;
}

/* Interpolated TSDF of any observed cell (no band requirement). */
int or_sample(const double* tsdf, const double* weight, const or_grid* g, const double q[3], double* val)
{
    return sample_cell(tsdf, weight, g, q, 0, val, 0);
}

/* Interpolated TSDF when the point falls in a valid cell (band required). */
int or_sample_band(const double* tsdf, const double* weight, const or_grid* g, const double q[3], double* val)
{
    return sample_cell(tsdf, weight, g, q, 1, val, 0);
}

/* validity of the cell with lower corner (i, j, k) */
static int cell_ok(const double* tsdf, const double* weight, const or_grid* g, long i, long j, long k)
{
    if (i < 0 || j < 0 || k < 0 || i > g->nx - 2 || j > g->ny - 2 || k > g->nz - 2) return 0;
    for (int c = 0; c < 8; ++c) {
        size_t idx = node_index(g, i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1));
        if (!(weight[idx] > 0.0) || !(fabs(tsdf[idx]) < 1.0)) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Fitness (Sec. III-B): E(T) = (1/|X|) sum_{x in X} |TSDF(T x)|, the TSDF   */
/* stored already divided by tau.  X = points falling in valid cells.        */
/* ------------------------------------------------------------------------ */

static void transform(const double T[12], const double x[3], double q[3])
{
    for (int r = 0; r < 3; ++r)
        q[r] = T[4 * r + 0] * x[0] + T[4 * r + 1] * x[1] + T[4 * r + 2] * x[2] + T[4 * r + 3];
}

/* One pose against points (every `stride`-th of n).  S = sum |tsdf|,
 * C = |X|.  Test aid: when amb != NULL, a point lying within eps_g voxels of
 * a cell face across which cell validity changes (its membership in X could
 * flip under a perturbation of that size) is counted in *amb instead of S, C
 * -- S and C then cover the unambiguous points only -- and the value it
 * contributes when counted as valid (its |tsdf| in the valid cell) is
 * written to vals[0 .. cap). */
static void fitness_one(const double* tsdf, const double* weight, const or_grid* g,
                        const double* pts, long n, long stride, const double T[12],
                        double* S, long* C, long* amb, double eps_g, double* vals, int cap)
{
    double s = 0.0;
    long c = 0, a = 0;
    for (long j = 0; j < n; j += stride) {
        double q[3], t, gc[3];
        transform(T, pts + 3 * j, q);
        int ok = sample_cell(tsdf, weight, g, q, 1, &t, gc);
        if (amb) {
            long i0[3];
            for (int ax = 0; ax < 3; ++ax) i0[ax] = (long)floor(gc[ax]);
            int here = cell_ok(tsdf, weight, g, i0[0], i0[1], i0[2]);
            int flag = 0;
            long alt[3] = {i0[0], i0[1], i0[2]};
            for (int ax = 0; ax < 3 && !flag; ++ax) {
                double fr = gc[ax] - floor(gc[ax]);
                alt[0] = i0[0];
                alt[1] = i0[1];
                alt[2] = i0[2];
                if (fr < eps_g) alt[ax] -= 1;
                else if (fr > 1.0 - eps_g) alt[ax] += 1;
                else continue;
                if (cell_ok(tsdf, weight, g, alt[0], alt[1], alt[2]) != here) flag = 1;
            }
            if (flag) {
                double v = 0.0;
                if (ok) {
                    v = fabs(t);
                } else {
                    /* the value in the neighbouring valid cell, at the face */
                    double qa[3];
                    for (int ax = 0; ax < 3; ++ax) {
                        double lo = (double)alt[ax], hi = lo + 1.0;
                        double gg = gc[ax] < lo ? lo : (gc[ax] > hi ? hi - 1e-12 : gc[ax]);
                        qa[ax] = g->origin[ax] + gg * g->voxel_size;
                    }
                    double ta;
                    if (sample_cell(tsdf, weight, g, qa, 1, &ta, 0)) v = fabs(ta);
                }
                if (a < cap) vals[a] = v;
                ++a;
                continue;
            }
        }
        if (ok) {
            s += fabs(t);
            c += 1;
        }
    }
    *S = s;
    *C = c;
    if (amb) *amb = a;
}

/* K poses (row-major 3x4) against the points: S_k, C_k, E_k (= +inf when
 * C_k = 0, reading: an empty valid set never improves the fit).  With amb,
 * see fitness_one: vals holds cap values per pose. */
void or_fitness(const double* tsdf, const double* weight, const or_grid* g,
                const double* pts, long n, long stride, const double* poses, int K,
                double* S, long* C, double* E, long* amb, double eps_g, double* vals, int cap)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        double s;
        long c, a = 0;
        fitness_one(tsdf, weight, g, pts, n, stride, poses + 12 * k, &s, &c, amb ? &a : 0, eps_g,
                    vals ? vals + (size_t)k * cap : 0, cap);
        S[k] = s;
        C[k] = c;
        E[k] = c > 0 ? s / (double)c : INFINITY;
        if (amb) amb[k] = a;
    }
}

/* ------------------------------------------------------------------------ */
/* SE(3) pieces used by the search                                           */
/* ------------------------------------------------------------------------ */

/* Rotation matrix of a rotation vector (Rodrigues' formula), row-major 3x3. */
void or_so3_exp(const double w[3], double R[9])
{
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double kk = 0.0;
            for (int m = 0; m < 3; ++m) kk += K[3 * r + m] * K[3 * m + c];
            R[3 * r + c] = (r == c ? 1.0 : 0.0) + a * K[3 * r + c] + b * kk;
        }
}

/* reading: a delta pose is [Exp(dw) | dt] (rotation and translation kept
 * apart, as the paper averages them separately).  compose_mode 0 applies it
 * on the left of the camera-to-world pose exactly as written, dP * P:
 * R' = dR R, t' = dR t + dt.  compose_mode 1 turns the camera about its own
 * centre instead: R' = dR R, t' = t + dt. */
static void compose(const double dR[9], const double dt[3], const double P[12], int mode, double out[12])
{
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += dR[3 * r + m] * P[4 * m + c];
            out[4 * r + c] = acc;
        }
        double tr = 0.0;
        if (mode == 0) {
            for (int m = 0; m < 3; ++m) tr += dR[3 * r + m] * P[4 * m + 3];
        } else {
            tr = P[4 * r + 3];
        }
        out[4 * r + 3] = tr + dt[r];
    }
}

/* Delta pose of template u scaled by the search size: rotation vector
 * omega * pi/180 * u[0:3] (radians), translation v / 100 * u[3:6] (metres). */
static void delta_of_template(const float* u, double s_deg, double s_cm, double dw[3], double dt[3])
{
    for (int a = 0; a < 3; ++a) {
        dw[a] = s_deg * OR_PI / 180.0 * (double)u[a];
        dt[a] = s_cm / 100.0 * (double)u[3 + a];
    }
}

/* The K global transforms dP_k * P of one iteration (row-major 3x4). */
void or_particles(const float* templ, int K, const double P[12], double s_deg, double s_cm,
                  int compose_mode, double* out)
{
    for (int k = 0; k < K; ++k) {
        double dw[3], dt[3], dR[9];
        delta_of_template(templ + 6 * k, s_deg, s_cm, dw, dt);
        or_so3_exp(dw, dR);
        compose(dR, dt, P, compose_mode, out + 12 * k);
    }
}

/* Gram-Schmidt on the rows of the rotation block. */
static void orthonormalise(double P[12])
{
    double r0[3] = {P[0], P[1], P[2]}, r1[3] = {P[4], P[5], P[6]};
    double n0 = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    for (int a = 0; a < 3; ++a) r0[a] /= n0;
    double d = r0[0] * r1[0] + r0[1] * r1[1] + r0[2] * r1[2];
    for (int a = 0; a < 3; ++a) r1[a] -= d * r0[a];
    double n1 = sqrt(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
    for (int a = 0; a < 3; ++a) r1[a] /= n1;
    double r2[3] = {r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2], r0[0] * r1[1] - r0[1] * r1[0]};
    for (int a = 0; a < 3; ++a) {
        P[a] = r0[a];
        P[4 + a] = r1[a];
        P[8 + a] = r2[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Randomized optimization (Sec. III-B) for one frame.                       */
/* Returns 0 when tracked, 1 when lost (then out = P0).                      */
/* ------------------------------------------------------------------------ */
int or_track(const double* tsdf, const double* weight, const or_grid* g,
             const float* depth, const or_intr* in, const or_params* prm,
             const float* templ, int k_max, const double P0[12], double out[12], or_stats* st)
{
    long npix = (long)in->width * in->height;
    double* pts = (double*)malloc(sizeof(double) * 3 * (size_t)(npix > 0 ? npix : 1));
    long n = or_backproject(depth, in, 1, pts);
    int kmax_used = 0;
    for (int a = 0; a < 3; ++a)
        if (prm->k_sched[a] > kmax_used) kmax_used = prm->k_sched[a];
    if (kmax_used > k_max) kmax_used = k_max;
    double* T = (double*)malloc(sizeof(double) * 12 * (size_t)kmax_used);
    double* S = (double*)malloc(sizeof(double) * (size_t)kmax_used);
    double* E = (double*)malloc(sizeof(double) * (size_t)kmax_used);
    long* C = (long*)malloc(sizeof(long) * (size_t)kmax_used);

    double P[12], s_deg = prm->s0_deg, s_cm = prm->s0_cm;
    memcpy(P, P0, sizeof(P));
    int lost = 0;
    if (st) {
        memset(st, 0, sizeof(*st));
        st->n_points = (int)n;
    }
    for (int it = 0; it < prm->n_iters && it < OR_MAX_ITERS; ++it) {
        int K = prm->k_sched[it % 3];
        if (K > k_max) K = k_max;
        int stride = prm->decim_sched[it % 3];
        long n_eval = n > 0 ? (n + stride - 1) / stride : 0;

        /* sample delta poses within s and form dP_k * P (particle 0 is P) */
        or_particles(templ, K, P, s_deg, s_cm, prm->compose_mode, T);
        or_fitness(tsdf, weight, g, pts, n, stride, T, K, S, C, E, 0, 0.0, 0, 0);

        /* best particle: smallest E, lowest index among equals */
        int kb = 0;
        for (int k = 1; k < K; ++k)
            if (E[k] < E[kb]) kb = k;
        double E0 = E[0];
        if (it == 0 && (!isfinite(E0) || (double)C[0] < prm->min_valid_frac * (double)n_eval)) {
            lost = 1;
            if (st) {
                st->E0[it] = E0;
                st->n_valid0[it] = (int)C[0];
                st->n_eval[it] = (int)n_eval;
                st->k_used[it] = K;
                st->s[it][0] = s_deg;
                st->s[it][1] = s_cm;
                st->n_iters = 1;
            }
            break;
        }

        /* advantage set {k : E_k < E(P)} and its mean delta pose */
        int n_adv = 0;
        double mw[3] = {0, 0, 0}, mt[3] = {0, 0, 0};
        double margin = INFINITY;
        for (int k = 1; k < K; ++k) {
            if (E[k] < E0) {
                double dw[3], dt[3];
                delta_of_template(templ + 6 * k, s_deg, s_cm, dw, dt);
                for (int a = 0; a < 3; ++a) {
                    mw[a] += dw[a];
                    mt[a] += dt[a];
                }
                ++n_adv;
            }
            if (isfinite(E[k]) && isfinite(E0) && E0 > 0.0) {
                double m = fabs(E[k] - E0) / E0;
                if (m < margin) margin = m;
            }
        }
        double second = INFINITY;
        for (int k = 0; k < K; ++k)
            if (k != kb && E[k] < second) second = E[k];
        double gap = (isfinite(E[kb]) && E[kb] > 0.0) ? (second - E[kb]) / E[kb] : INFINITY;

        double Pn[12], E_new;
        if (prm->update_mode == 0) {
            if (n_adv > 0) {
                for (int a = 0; a < 3; ++a) {
                    mw[a] /= (double)n_adv;
                    mt[a] /= (double)n_adv;
                }
                double dR[9];
                or_so3_exp(mw, dR);
                compose(dR, mt, P, prm->compose_mode, Pn);
                orthonormalise(Pn);
                double s1, e1;
                long c1;
                or_fitness(tsdf, weight, g, pts, n, stride, Pn, 1, &s1, &c1, &e1, 0, 0.0, 0, 0);
                E_new = e1;
            } else {
                memcpy(Pn, P, sizeof(Pn));
                E_new = E0;
            }
        } else {
            memcpy(Pn, T + 12 * kb, sizeof(Pn));
            orthonormalise(Pn);
            E_new = E[kb];
        }
        if (st) {
            st->E0[it] = E0;
            st->E_best[it] = E[kb];
            st->E_new[it] = E_new;
            st->best[it] = kb;
            st->n_adv[it] = n_adv;
            st->n_valid0[it] = (int)C[0];
            st->n_eval[it] = (int)n_eval;
            st->k_used[it] = K;
            st->s[it][0] = s_deg;
            st->s[it][1] = s_cm;
            memcpy(st->pose[it], Pn, sizeof(Pn));
            st->adv_margin[it] = margin;
            st->best_gap[it] = gap;
            st->n_iters = it + 1;
        }
        memcpy(P, Pn, sizeof(P));
        /* search size: s <- beta s + (1 - beta) E(P) s; reading: an empty
         * valid set (E = +inf) leaves s unchanged */
        double e = isfinite(E_new) ? E_new : 1.0;
        double fct = prm->beta + (1.0 - prm->beta) * e;
        s_deg *= fct;
        s_cm *= fct;
    }
    if (lost) memcpy(out, P0, sizeof(double) * 12);
    else memcpy(out, P, sizeof(double) * 12);
    if (st) st->lost = lost;
    free(pts);
    free(T);
    free(S);
    free(E);
    free(C);
    return lost;
}

/* ------------------------------------------------------------------------ */
/* Alignment loss and its derivatives (gradient refinement of a pose found  */
/* by the search; the residual is the TSDF of Sec. III-B, squared).          */
/* ------------------------------------------------------------------------ */
/* reading: the loss of pose T over points x_j is L(T) = sum over the points
 * falling in valid cells of tsdf(T x_j)^2 (tsdf normalised by tau, validity
 * as in the fitness).  A pose is perturbed as
 *     q = Exp(omega) (R x + t) + v,       xi = (omega, v),
 * so dq/dv = I and, with Exp(omega + d) = Exp(J_l(omega) d) Exp(omega) (J_l
 * the left Jacobian of SO(3)), dq/domega = -[q - v]x J_l(omega); at xi = 0
 * this is the usual left perturbation dq/dxi = [-[q]x | I].  With grad t the
 * gradient of the trilinear interpolant in metres:
 *     dL/dv     = sum 2 t grad t,
 *     dL/domega = J_l(omega)^T sum 2 t ((q - v) x grad t).
 * dL/dV_n = sum 2 t w_n(q) over the samples whose cell has node n (w_n its
 * trilinear weight): the derivative with respect to the stored tsdf value of
 * node n, at fixed cell validity. */

/* value, gradient in grid units (d t / d g), lower cell corner and
 * fractions of the valid cell containing q; 0 when q is in no valid cell */
static int sample_grad(const double* tsdf, const double* weight, const or_grid* g, const double q[3],
                       double* val, double dg[3], long i0[3], double f[3], double v[8])
{
    double gc[3];
    int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        gc[a] = (q[a] - g->origin[a]) / g->voxel_size;
        if (!(gc[a] >= 0.0 && gc[a] < (double)(n[a] - 1))) return 0;
        i0[a] = (long)floor(gc[a]);
        f[a] = gc[a] - (double)i0[a];
    }
    for (int c = 0; c < 8; ++c) {
        size_t idx = node_index(g, i0[0] + (c & 1), i0[1] + ((c >> 1) & 1), i0[2] + ((c >> 2) & 1));
        if (!(weight[idx] > 0.0) || !(fabs(tsdf[idx]) < 1.0)) return 0;
        v[c] = tsdf[idx];
    }
    double x00 = v[0] + f[0] * (v[1] - v[0]);
    double x10 = v[2] + f[0] * (v[3] - v[2]);
    double x01 = v[4] + f[0] * (v[5] - v[4]);
    double x11 = v[6] + f[0] * (v[7] - v[6]);
    double y0 = x00 + f[1] * (x10 - x00);
    double y1 = x01 + f[1] * (x11 - x01);
    *val = y0 + f[2] * (y1 - y0);
    /* partial derivatives of the nested linear interpolations */
    double dx00 = v[1] - v[0], dx10 = v[3] - v[2], dx01 = v[5] - v[4], dx11 = v[7] - v[6];
    double dy0 = dx00 + f[1] * (dx10 - dx00), dy1 = dx01 + f[1] * (dx11 - dx01);
    dg[0] = dy0 + f[2] * (dy1 - dy0);
    dg[1] = (x10 - x00) + f[2] * ((x11 - x01) - (x10 - x00));
    dg[2] = y1 - y0;
    return 1;
}

/* left Jacobian of SO(3): I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2 */
static void so3_left_jacobian(const double w[3], double J[9])
{
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b;
    if (th < 1e-6) {
        a = 0.5 - th2 / 24.0;
        b = 1.0 / 6.0 - th2 / 120.0;
    } else {
        a = (1.0 - cos(th)) / th2;
        b = (th - sin(th)) / (th2 * th);
    }
    double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double kk = 0.0;
            for (int m = 0; m < 3; ++m) kk += K[3 * r + m] * K[3 * m + c];
            J[3 * r + c] = (r == c ? 1.0 : 0.0) + a * K[3 * r + c] + b * kk;
        }
}

/* The pose q = Exp(omega) (R x + t) + v as a row-major 3x4 transform. */
void or_perturb_pose(const double T[12], const double xi[6], double out[12])
{
    double dR[9];
    or_so3_exp(xi, dR);
    compose(dR, xi + 3, T, 0, out);
}

/* Loss, valid count, dL/dxi (6) at xi, and dL/dV accumulated into gV
 * (n_nodes, may be NULL) for one pose T perturbed by xi (may be NULL). */
void or_align_loss(const double* tsdf, const double* weight, const or_grid* g, const double* pts, long n,
                   const double T[12], const double* xi, double* L, long* C, double grad_xi[6], double* gV)
{
    double Tp[12], zero[6] = {0, 0, 0, 0, 0, 0};
    const double* x6 = xi ? xi : zero;
    or_perturb_pose(T, x6, Tp);
    double loss = 0.0, gw[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
    long c = 0;
    for (long j = 0; j < n; ++j) {
        double q[3], t, dg[3], f[3], v[8];
        long i0[3];
        transform(Tp, pts + 3 * j, q);
        if (!sample_grad(tsdf, weight, g, q, &t, dg, i0, f, v)) continue;
        loss += t * t;
        c += 1;
        double gt[3] = {dg[0] / g->voxel_size, dg[1] / g->voxel_size, dg[2] / g->voxel_size};
        double r[3] = {q[0] - x6[3], q[1] - x6[4], q[2] - x6[5]};
        double cr[3] = {r[1] * gt[2] - r[2] * gt[1], r[2] * gt[0] - r[0] * gt[2], r[0] * gt[1] - r[1] * gt[0]};
        for (int a = 0; a < 3; ++a) {
            gw[a] += 2.0 * t * cr[a];
            gv[a] += 2.0 * t * gt[a];
        }
        if (gV)
            for (int cc = 0; cc < 8; ++cc) {
                double w = ((cc & 1) ? f[0] : 1.0 - f[0]) * (((cc >> 1) & 1) ? f[1] : 1.0 - f[1]) *
                           (((cc >> 2) & 1) ? f[2] : 1.0 - f[2]);
                gV[node_index(g, i0[0] + (cc & 1), i0[1] + ((cc >> 1) & 1), i0[2] + ((cc >> 2) & 1))] +=
                    2.0 * t * w;
            }
    }
    double J[9];
    so3_left_jacobian(x6, J);
    for (int a = 0; a < 3; ++a) {
        grad_xi[a] = J[a] * gw[0] + J[3 + a] * gw[1] + J[6 + a] * gw[2];  /* J^T gw */
        grad_xi[3 + a] = gv[a];
    }
    *L = loss;
    *C = c;
}

/* reading: the refinement after the search is a damped Gauss-Newton
 * (Levenberg-Marquardt) on the residuals r_j = tsdf(T x_j) over the valid
 * points: J_j = grad t^T [-[q]x | I], H = sum J_j^T J_j, b = sum J_j^T r_j;
 * the step solves (H + lambda diag(H)) d = -b and the candidate is
 * [Exp(d_omega) | d_v] applied on the left of T.  The objective is the mean
 * squared residual over the valid points; a candidate is accepted only when
 * it lowers it (then lambda /= 10), otherwise it is dropped and
 * lambda *= 10.  lambda starts at 1e-3; `steps` candidates are tried.
 * trace[0] = objective at T, trace[s] = objective after step s.  Returns the
 * number of accepted steps; T is updated in place. */
static void gn_system(const double* tsdf, const double* weight, const or_grid* g, const double* pts, long n,
                      const double T[12], double H[36], double b[6], double* L, long* C)
{
    memset(H, 0, 36 * sizeof(double));
    memset(b, 0, 6 * sizeof(double));
    double loss = 0.0;
    long c = 0;
    for (long j = 0; j < n; ++j) {
        double q[3], t, dg[3], f[3], v[8];
        long i0[3];
        transform(T, pts + 3 * j, q);
        if (!sample_grad(tsdf, weight, g, q, &t, dg, i0, f, v)) continue;
        double gt[3] = {dg[0] / g->voxel_size, dg[1] / g->voxel_size, dg[2] / g->voxel_size};
        double Jr[6] = {q[1] * gt[2] - q[2] * gt[1], q[2] * gt[0] - q[0] * gt[2], q[0] * gt[1] - q[1] * gt[0],
                        gt[0], gt[1], gt[2]};
        for (int r = 0; r < 6; ++r) {
            b[r] += Jr[r] * t;
            for (int cc = 0; cc < 6; ++cc) H[6 * r + cc] += Jr[r] * Jr[cc];
        }
        loss += t * t;
        c += 1;
    }
    *L = loss;
    *C = c;
}

/* solve the 6x6 system A d = y by Gaussian elimination with partial
 * pivoting; 0 when singular */
static int solve6(const double A_in[36], const double y_in[6], double d[6])
{
    double A[36], y[6];
    memcpy(A, A_in, sizeof(A));
    memcpy(y, y_in, sizeof(y));
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        for (int r = col + 1; r < 6; ++r)
            if (fabs(A[6 * r + col]) > fabs(A[6 * piv + col])) piv = r;
        if (!(fabs(A[6 * piv + col]) > 0.0)) return 0;
        if (piv != col) {
            for (int cc = 0; cc < 6; ++cc) {
                double tmp = A[6 * col + cc];
                A[6 * col + cc] = A[6 * piv + cc];
                A[6 * piv + cc] = tmp;
            }
            double tmp = y[col];
            y[col] = y[piv];
            y[piv] = tmp;
        }
        for (int r = col + 1; r < 6; ++r) {
            double m = A[6 * r + col] / A[6 * col + col];
            for (int cc = col; cc < 6; ++cc) A[6 * r + cc] -= m * A[6 * col + cc];
            y[r] -= m * y[col];
        }
    }
    for (int r = 5; r >= 0; --r) {
        double acc = y[r];
        for (int cc = r + 1; cc < 6; ++cc) acc -= A[6 * r + cc] * d[cc];
        d[r] = acc / A[6 * r + r];
    }
    return 1;
}

int or_polish(const double* tsdf, const double* weight, const or_grid* g, const double* pts, long n,
              double T[12], int steps, double* trace)
{
    double H[36], b[6], L;
    long C;
    double lambda = 1e-3;
    int accepted = 0;
    gn_system(tsdf, weight, g, pts, n, T, H, b, &L, &C);
    double obj = C > 0 ? L / (double)C : INFINITY;
    if (trace) trace[0] = obj;
    for (int st = 0; st < steps; ++st) {
        double A[36], y[6], d[6], Tc[12];
        int ok = C > 0;
        if (ok) {
            for (int r = 0; r < 36; ++r) A[r] = H[r];
            for (int r = 0; r < 6; ++r) {
                A[7 * r] += lambda * H[7 * r];
                y[r] = -b[r];
            }
            ok = solve6(A, y, d);
        }
        if (ok) {
            or_perturb_pose(T, d, Tc);
            double Hc[36], bc[6], Lc;
            long Cc;
            gn_system(tsdf, weight, g, pts, n, Tc, Hc, bc, &Lc, &Cc);
            double objc = Cc > 0 ? Lc / (double)Cc : INFINITY;
            if (objc < obj) {
                memcpy(T, Tc, sizeof(Tc));
                memcpy(H, Hc, sizeof(Hc));
                memcpy(b, bc, sizeof(bc));
                L = Lc;
                C = Cc;
                obj = objc;
                lambda /= 10.0;
                ++accepted;
            } else {
                lambda *= 10.0;
            }
        }
        if (trace) trace[st + 1] = obj;
    }
    return accepted;
}

/* ------------------------------------------------------------------------ */
/* Fusion "the same as KinectFusion" (Sec. III): projective TSDF update.     */
/* ------------------------------------------------------------------------ */
/* reading: for node X_w, X_c = R^T (X_w - t); with z_c > 0 it projects to
 * the nearest pixel (floor(u + 1/2), floor(v + 1/2)); with a usable depth d
 * there, sdf = d - z_c; nodes with sdf >= -tau take t = min(1, sdf / tau)
 * into the running average tsdf <- (w tsdf + t) / (w + 1), and
 * w <- min(w + 1, max_weight).  Unobserved nodes have w = 0.
 * If mask != NULL, mask[node] = 1 marks nodes whose update could change
 * under a perturbation of eps_px pixels or eps_m metres (test aid); the
 * function returns their count. */
long or_integrate(double* tsdf, double* weight, const or_grid* g, const float* depth,
                  const or_intr* in, const double pose[12], unsigned char* mask,
                  double eps_px, double eps_m)
{
    const double* R = pose;  /* row-major 3x4 */
    long amb = 0;
#pragma omp parallel for schedule(static) reduction(+ : amb)
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                size_t idx = node_index(g, i, j, k);
                double X[3] = {g->origin[0] + g->voxel_size * (double)i, g->origin[1] + g->voxel_size * (double)j,
                               g->origin[2] + g->voxel_size * (double)k};
                double d[3] = {X[0] - R[3], X[1] - R[7], X[2] - R[11]};
                double xc = R[0] * d[0] + R[4] * d[1] + R[8] * d[2];
                double yc = R[1] * d[0] + R[5] * d[1] + R[9] * d[2];
                double zc = R[2] * d[0] + R[6] * d[1] + R[10] * d[2];
                if (mask) mask[idx] = 0;
                /* a node within eps_m of the camera plane may fall on either
                 * side of z = 0 */
                if (mask && fabs(zc) < eps_m) {
                    mask[idx] = 1;
                    ++amb;
                }
                if (!(zc > 0.0)) continue;
                double u = in->fx * xc / zc + in->cx;
                double v = in->fy * yc / zc + in->cy;
                if (mask && !mask[idx]) {
                    double fu = u + 0.5 - floor(u + 0.5), fv = v + 0.5 - floor(v + 0.5);
                    int near_u = fu < eps_px || fu > 1.0 - eps_px;
                    int near_v = fv < eps_px || fv > 1.0 - eps_px;
                    int inside = u > -1.5 && u < in->width + 0.5 && v > -1.5 && v < in->height + 0.5;
                    if (inside && (near_u || near_v)) {
                        mask[idx] = 1;
                        ++amb;
                    }
                }
                double uf = floor(u + 0.5), vf = floor(v + 0.5);
                if (!(uf >= 0.0 && uf < (double)in->width && vf >= 0.0 && vf < (double)in->height)) continue;
                float dz = depth[(size_t)vf * in->width + (size_t)uf];
                if (!depth_valid(dz, in)) continue;
                double sdf = (double)dz - zc;
                if (mask && !mask[idx] && fabs(sdf + g->trunc) < eps_m) {
                    mask[idx] = 1;
                    ++amb;
                }
                if (sdf < -g->trunc) continue;
                double t = sdf / g->trunc;
                if (t > 1.0) t = 1.0;
                double w = weight[idx];
                tsdf[idx] = (w * tsdf[idx] + t) / (w + 1.0);
                weight[idx] = (w + 1.0 < (double)g->max_weight) ? w + 1.0 : (double)g->max_weight;
            }
    return amb;
}

/* ------------------------------------------------------------------------ */
/* Raycast of the fused TSDF (for views and tests).                          */
/* ------------------------------------------------------------------------ */
/* reading: march the pixel's ray at camera depths z_i = depth_min + i * step
 * up to depth_max; the first pair of consecutive usable samples going from
 * positive to non-positive brackets the surface, located by linear
 * interpolation; the output is that camera depth (0 when nothing is hit) and
 * the unit gradient of the interpolated field there (central differences at
 * +-voxel/2 along the world axes; NaN when a sample is unusable). */
void or_raycast(const double* tsdf, const double* weight, const or_grid* g, const or_intr* in,
                const double pose[12], double step, double* depth_out, double* normal_out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < in->height; ++v)
        for (int u = 0; u < in->width; ++u) {
            double dc[3] = {((double)u - in->cx) / in->fx, ((double)v - in->cy) / in->fy, 1.0};
            double dw[3], o[3];
            for (int r = 0; r < 3; ++r) {
                dw[r] = pose[4 * r] * dc[0] + pose[4 * r + 1] * dc[1] + pose[4 * r + 2] * dc[2];
                o[r] = pose[4 * r + 3];
            }
            size_t pix = (size_t)v * in->width + u;
            double hit = 0.0;
            int have_prev = 0;
            double prev = 0.0;
            long nsteps = (long)floor((in->depth_max - in->depth_min) / step);
            for (long i = 0; i <= nsteps; ++i) {
                double z = in->depth_min + (double)i * step;
                double q[3] = {o[0] + z * dw[0], o[1] + z * dw[1], o[2] + z * dw[2]};
                double t;
                if (!or_sample(tsdf, weight, g, q, &t)) {
                    have_prev = 0;
                    continue;
                }
                if (have_prev && prev > 0.0 && t <= 0.0) {
                    hit = (z - step) + step * prev / (prev - t);
                    break;
                }
                prev = t;
                have_prev = 1;
            }
            depth_out[pix] = hit;
            if (normal_out) {
                double nrm[3] = {NAN, NAN, NAN};
                if (hit > 0.0) {
                    double q[3] = {o[0] + hit * dw[0], o[1] + hit * dw[1], o[2] + hit * dw[2]};
                    double h = 0.5 * g->voxel_size, gr[3];
                    int ok = 1;
                    for (int a = 0; a < 3 && ok; ++a) {
                        double qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]}, tp, tm;
                        qp[a] += h;
                        qm[a] -= h;
                        ok = or_sample(tsdf, weight, g, qp, &tp) && or_sample(tsdf, weight, g, qm, &tm);
                        gr[a] = tp - tm;
                    }
                    if (ok) {
                        double len = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
                        if (len > 0.0)
                            for (int a = 0; a < 3; ++a) nrm[a] = gr[a] / len;
                    }
                }
                for (int a = 0; a < 3; ++a) normal_out[3 * pix + a] = nrm[a];
            }
        }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
