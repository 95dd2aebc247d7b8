/*
 * mvtsdf_oracle.c -- plain FP64 CPU oracle for multi-volume projective TSDF
 * integration and raycasting, written from Salvato, Finman and Leonard,
 * "Multi-Volume High Resolution RGB-D Mapping with Dynamic Volume Placement"
 * (arXiv 1511.07106).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * library; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA path.  Everything is computed in double precision, voxel by
 * voxel and ray by ray, in the order the paper states the steps; there is no
 * blocking, no bricking and no empty-space skipping here.
 *
 * Readings of the paper that this file fixes (the paper is silent or
 * garbled at these points):
 *   - voxel i of a volume with lattice offset h_t sits at world position
 *     (h_t + i) * s, s = voxel pitch (Sec. Volumetric Integration, t_s = t_l + h_t;
 *     Sec. Dynamic Mapping for SLAM, h_t on an integer lattice);
 *   - the pose T = [R|t] maps camera to world (Sec. Depth Map Conversion);
 *   - the measured distance of a voxel is the projective distance along its
 *     ray seen from the current camera: sdf = (D - z) * |p_c| / z
 *     (Sec. Volumetric Integration, dist = D - d_m, read with d_m measured
 *     from the camera of the current frame);
 *   - truncation: voxels with sdf < -mu are not updated, otherwise
 *     f = min(1, sdf / mu) in units of mu;
 *   - weights grow by one per frame up to a cap: per-frame weight 1,
 *     F' = (F W + f) / (W + 1), W' = min(W + 1, W_max);
 *   - colour (the paper shows coloured models but gives no rule): a running
 *     average inside the band |sdf| < mu, rounded half up, colour weight in
 *     the alpha byte capped at color_w_max;
 *   - raycast (Sec. Raycasting, Algorithm 1): the ray of pixel (x, y) is
 *     o = t, d = R K^-1 [x y 1]^T, so the ray parameter tau is z-depth.
 *     Samples sit on the global grid tau_k = k * Delta with
 *     Delta = step * s / |d| (same grid in every volume of equal pitch).
 *     A sample is valid when the 8 corners of its trilinear cell have W > 0.
 *     The first pair of consecutive valid samples with F > 0 then F <= 0
 *     brackets the surface; an invalid sample breaks the pair.  The root of
 *     the trilinear interpolant inside the bracket is found by bisection.
 *   - normal = normalised analytic gradient of the trilinear interpolant in
 *     the hit cell (the TSDF derivative at the zero crossing);
 *     colour = trilinear RGB in the hit cell, rounded half up;
 *   - all volumes write one map; the smallest ray distance wins, exact ties
 *     go to the lower volume id (Sec. Raycasting, last paragraph).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

typedef struct {
    int32_t h[3];   /* lattice offset h_t, voxels */
    int32_t r[3];   /* voxels per axis h_r */
    double s;       /* voxel pitch, metres */
    double *F;      /* r0*r1*r2 normalised TSDF, x fastest */
    double *W;      /* r0*r1*r2 weights */
    uint8_t *rgba;  /* 4 per voxel (A = colour weight), may be NULL */
} orc_volume;

typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
} orc_intrinsics;

typedef struct {
    double trunc_vox;      /* truncation mu, in voxels */
    double w_max;          /* weight cap */
    int32_t color_w_max;   /* colour weight cap, <= 255 */
    double z_min, z_max;   /* valid depth / ray range, metres */
    double step_vox;       /* raycast sample spacing, voxels (<= 1) */
    /* decision margins: outputs whose FP64 decision lies closer than these
     * to a threshold are flagged (an FP32 implementation may decide them
     * the other way). */
    double eps_px;         /* pixel rounding, pixels */
    double eps_sdf;        /* sdf thresholds, fraction of mu */
    double eps_z;          /* camera z near 0, metres */
    double eps_f;          /* sign of a ray sample, TSDF units */
    double eps_q;          /* cell boundary, voxels */
    double eps_tau;        /* sample-range endpoints, fraction of Delta */
} orc_config;

/* per-voxel integration flags */
enum { ORC_IF_Z = 1, ORC_IF_PIX = 2, ORC_IF_GATE = 4, ORC_IF_BAND = 8 };
/* per-pixel raycast flags */
enum { ORC_RF_SIGN = 1, ORC_RF_CELL = 2, ORC_RF_RANGE = 4, ORC_RF_FACE = 8,
       ORC_RF_TIE = 16, ORC_RF_GRAD = 32 };

static size_t vox_index(const orc_volume *v, int64_t x, int64_t y, int64_t z)
{
    return ((size_t)z * (size_t)v->r[1] + (size_t)y) * (size_t)v->r[0] + (size_t)x;
}

static int near_half_integer_boundary(double u, double eps)
{
    /* nearest-pixel rounding floor(u + 1/2) changes where u + 1/2 is an integer */
    double w = u + 0.5;
    double fl = floor(w);
    return (w - fl) < eps || (fl + 1.0 - w) < eps;
}

/* ------------------------------------------------------------------------ */
/* Volumetric integration (Sec. Volumetric Integration; Algorithm 1, first  */
/* double loop).  One voxel.                                                */
/* ------------------------------------------------------------------------ */
static void integrate_voxel(orc_volume *v, int64_t x, int64_t y, int64_t z,
                            const float *depth, const uint8_t *rgb,
                            const orc_intrinsics *K, const double R[9], const double t[3],
                            const orc_config *c, uint8_t *flag, int64_t cnt[2])
{
    uint8_t fl = 0;
    /* t_s = t_l + h_t, in metres */
    const double pw[3] = { (double)(v->h[0] + x) * v->s,
                           (double)(v->h[1] + y) * v->s,
                           (double)(v->h[2] + z) * v->s };
    const double dw[3] = { pw[0] - t[0], pw[1] - t[1], pw[2] - t[2] };
    /* camera coordinates p_c = R^T (p_w - t) */
    const double X = R[0] * dw[0] + R[3] * dw[1] + R[6] * dw[2];
    const double Y = R[1] * dw[0] + R[4] * dw[1] + R[7] * dw[2];
    const double Z = R[2] * dw[0] + R[5] * dw[1] + R[8] * dw[2];
    const size_t i = vox_index(v, x, y, z);

    if (fabs(Z) < c->eps_z) fl |= ORC_IF_Z;
    if (!(Z > 0.0)) goto done;

    /* project to the image and take the nearest pixel */
    const double u = K->fx * X / Z + K->cx;
    const double w = K->fy * Y / Z + K->cy;
    if (near_half_integer_boundary(u, c->eps_px) || near_half_integer_boundary(w, c->eps_px))
        fl |= ORC_IF_PIX;
    const double ui = floor(u + 0.5), vi = floor(w + 0.5);
    if (ui < 0.0 || vi < 0.0 || ui >= (double)K->width || vi >= (double)K->height) goto done;
    const size_t pix = (size_t)vi * (size_t)K->width + (size_t)ui;

    const double D = (double)depth[pix];
    if (!(D > 0.0) || D < c->z_min || D > c->z_max) goto done;

    /* projective signed distance along the voxel's ray */
    const double norm_pc = sqrt(X * X + Y * Y + Z * Z);
    const double sdf = (D - Z) * (norm_pc / Z);
    const double mu = c->trunc_vox * v->s;
    if (fabs(sdf + mu) < c->eps_sdf * mu) fl |= ORC_IF_GATE;
    if (fabs(fabs(sdf) - mu) < c->eps_sdf * mu) fl |= ORC_IF_BAND;
    if (sdf < -mu) goto done;

    double f = sdf / mu;
    if (f > 1.0) f = 1.0;

    /* weighted running average with per-frame weight 1 and capped weight */
    const double Wold = v->W[i];
    v->F[i] = (v->F[i] * Wold + f) / (Wold + 1.0);
    v->W[i] = (Wold + 1.0 < c->w_max) ? Wold + 1.0 : c->w_max;
    cnt[0] += 1;

    if (rgb && v->rgba && fabs(sdf) < mu) {
        uint8_t *cv = v->rgba + 4 * i;
        const int64_t wc = cv[3];
        for (int ch = 0; ch < 3; ++ch) {
            const int64_t num = (int64_t)cv[ch] * wc + (int64_t)rgb[3 * pix + ch];
            /* round half up of num / (wc + 1), in integers */
            cv[ch] = (uint8_t)((2 * num + wc + 1) / (2 * (wc + 1)));
        }
        cv[3] = (uint8_t)((wc + 1 < c->color_w_max) ? wc + 1 : c->color_w_max);
        cnt[1] += 1;
    }
done:
    if (flag) flag[i] = fl;
}

static void pose_split(const double T[16], double R[9], double t[3])
{
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) R[3 * a + b] = T[4 * a + b];
        t[a] = T[4 * a + 3];
    }
}

/* Integrate one depth (+ optional RGB) frame into one volume.
 * depth: height*width float32 z-depth in metres (<= 0 or NaN = invalid).
 * rgb:   height*width*3 uint8 registered to depth, or NULL.
 * T:     4x4 row-major camera-to-world pose.
 * flags: per-voxel decision flags (ORC_IF_*), or NULL.
 * counts[0] += updated voxels, counts[1] += colour (band) voxels. */
ORC_EXPORT void orc_integrate(orc_volume *v, const float *depth, const uint8_t *rgb,
                              const orc_intrinsics *K, const double T[16],
                              const orc_config *c, uint8_t *flags, int64_t counts[2])
{
    double R[9], t[3];
    pose_split(T, R, t);
    int64_t tot0 = 0, tot1 = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : tot0, tot1)
    for (int64_t z = 0; z < v->r[2]; ++z) {
        int64_t cnt[2] = {0, 0};
        for (int64_t y = 0; y < v->r[1]; ++y)
            for (int64_t x = 0; x < v->r[0]; ++x)
                integrate_voxel(v, x, y, z, depth, rgb, K, R, t, c, flags, cnt);
        tot0 += cnt[0];
        tot1 += cnt[1];
    }
    if (counts) { counts[0] += tot0; counts[1] += tot1; }
}

/* The same update restricted to a list of voxels (linear indices, x
 * fastest); used to check large volumes on a sample. */
ORC_EXPORT void orc_integrate_voxels(orc_volume *v, const int64_t *idx, int64_t n,
                                     const float *depth, const uint8_t *rgb,
                                     const orc_intrinsics *K, const double T[16],
                                     const orc_config *c, uint8_t *flags, int64_t counts[2])
{
    double R[9], t[3];
    pose_split(T, R, t);
    int64_t cnt[2] = {0, 0};
    const int64_t rx = v->r[0], ry = v->r[1];
    for (int64_t j = 0; j < n; ++j) {
        const int64_t li = idx[j];
        const int64_t x = li % rx, y = (li / rx) % ry, z = li / (rx * ry);
        integrate_voxel(v, x, y, z, depth, rgb, K, R, t, c, flags, cnt);
    }
    if (counts) { counts[0] += cnt[0]; counts[1] += cnt[1]; }
}

/* ------------------------------------------------------------------------ */
/* Raycasting (Sec. Raycasting; Algorithm 1, pixel loop).                   */
/* ------------------------------------------------------------------------ */

/* trilinear cell of a point given in GLOBAL voxel coordinates g (the
 * paper's t_r; volume coordinates are t_r' = t_r - h_t): the lattice cell
 * floor(g), shifted into the volume and clamped so that the cell's upper
 * corner stays inside it.  Taking floor() before subtracting h_t makes the
 * choice of cell independent of which volume evaluates the point. */
static void cell_of(const orc_volume *v, const double g[3], int64_t cell[3], double fr[3])
{
    for (int a = 0; a < 3; ++a) {
        double fl = floor(g[a]) - (double)v->h[a];
        if (fl < 0.0) fl = 0.0;
        if (fl > (double)(v->r[a] - 2)) fl = (double)(v->r[a] - 2);
        cell[a] = (int64_t)fl;
        fr[a] = g[a] - (fl + (double)v->h[a]);
    }
}

static int cell_valid(const orc_volume *v, const int64_t cell[3])
{
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                if (!(v->W[vox_index(v, cell[0] + dx, cell[1] + dy, cell[2] + dz)] > 0.0))
                    return 0;
    return 1;
}

/* trilinear interpolation of F in a given cell; optional analytic gradient
 * (per voxel) */
static double trilinear_in_cell(const orc_volume *v, const int64_t cell[3], const double fr[3],
                                double grad[3])
{
    double c[2][2][2];
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                c[dz][dy][dx] = v->F[vox_index(v, cell[0] + dx, cell[1] + dy, cell[2] + dz)];
    const double x = fr[0], y = fr[1], z = fr[2];
    double val = 0.0;
    double g[3] = {0.0, 0.0, 0.0};
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const double wx = dx ? x : 1.0 - x;
                const double wy = dy ? y : 1.0 - y;
                const double wz = dz ? z : 1.0 - z;
                const double cv = c[dz][dy][dx];
                val += wx * wy * wz * cv;
                g[0] += (dx ? 1.0 : -1.0) * wy * wz * cv;
                g[1] += wx * (dy ? 1.0 : -1.0) * wz * cv;
                g[2] += wx * wy * (dz ? 1.0 : -1.0) * cv;
            }
    if (grad) { grad[0] = g[0]; grad[1] = g[1]; grad[2] = g[2]; }
    return val;
}

static uint8_t sample_flags(const orc_volume *v, const double q[3], int valid, double F,
                            const orc_config *c)
{
    uint8_t fl = 0;
    if (valid && fabs(F) < c->eps_f) fl |= ORC_RF_SIGN;
    /* near a cell boundary: would the cell on the other side give another
     * validity?  (the interpolant itself is continuous across the face) */
    for (int a = 0; a < 3; ++a) {
        const double fq = floor(q[a]);
        const double below = q[a] - fq, above = fq + 1.0 - q[a];
        if (below >= c->eps_q && above >= c->eps_q) continue;
        double q2[3] = {q[0], q[1], q[2]};
        q2[a] = (below < c->eps_q) ? fq - 0.5 * c->eps_q : fq + 1.0 + 0.5 * c->eps_q;
        int64_t cell2[3];
        double fr2[3];
        cell_of(v, q2, cell2, fr2);
        if (cell_valid(v, cell2) != valid) fl |= ORC_RF_CELL;
    }
    return fl;
}

typedef struct {
    int hit;
    double tau;
    double grad[3];
    int cell_ok;
    double rgb[3];
    uint8_t flags;
} orc_hit;

/* mark the 8 corners of a cell in a bitmap of the volume's voxels */
static void mark_cell(const orc_volume *v, const int64_t cell[3], uint64_t *bits)
{
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const size_t i = vox_index(v, cell[0] + dx, cell[1] + dy, cell[2] + dz);
                __atomic_fetch_or(&bits[i >> 6], (uint64_t)1 << (i & 63), __ATOMIC_RELAXED);
            }
}

/* march one ray through one volume.  touched / touched_rgb (bitmaps over
 * the volume's voxels, may be NULL) receive the voxels whose (F, W) the
 * march reads -- the corners of every sample's cell and of every bisection
 * midpoint's cell -- and the voxels whose colour the hit reads. */
static orc_hit march_volume_marking(const orc_volume *v, const double o[3], const double d[3],
                                    const orc_config *c, uint64_t *touched, uint64_t *touched_rgb)
{
    orc_hit out;
    memset(&out, 0, sizeof(out));
    const double s = v->s;
    /* ray in global voxel coordinates: g(tau) = q0 + tau * dv */
    double q0[3], dv[3];
    for (int a = 0; a < 3; ++a) {
        q0[a] = o[a] / s;
        dv[a] = d[a] / s;
    }
    /* interpolation domain [h_t, h_t + r - 1] per axis */
    double lo = c->z_min, hi = c->z_max;
    for (int a = 0; a < 3; ++a) {
        const double bmin = (double)v->h[a], bmax = (double)(v->h[a] + v->r[a] - 1);
        if (dv[a] == 0.0) {
            if (q0[a] < bmin || q0[a] > bmax) return out;
            continue;
        }
        double t0 = (bmin - q0[a]) / dv[a], t1 = (bmax - q0[a]) / dv[a];
        if (t0 > t1) { const double tmp = t0; t0 = t1; t1 = tmp; }
        if (t0 > lo) lo = t0;
        if (t1 < hi) hi = t1;
    }
    if (!(lo <= hi)) return out;
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double Delta = c->step_vox * s / dn;
    const double k0f = ceil(lo / Delta), k1f = floor(hi / Delta);
    {
        /* an endpoint within eps of a grid sample may include or exclude that
         * sample in another precision; an endpoint at tau = 0 (the camera) is
         * exact in every precision */
        const double a = lo / Delta, b = hi / Delta;
        if ((a != 0.0 && fabs(a - floor(a + 0.5)) < c->eps_tau) ||
            (b != 0.0 && fabs(b - floor(b + 0.5)) < c->eps_tau))
            out.flags |= ORC_RF_RANGE;
    }
    int state = 0; /* 0 none, 1 previous valid sample > 0, -1 previous valid sample <= 0 */
    double tau_prev = 0.0;
    for (double kf = k0f; kf <= k1f; kf += 1.0) {
        const double tau = kf * Delta;
        double q[3];
        for (int a = 0; a < 3; ++a) q[a] = q0[a] + tau * dv[a];
        int64_t cell[3];
        double fr[3];
        cell_of(v, q, cell, fr);
        if (touched) mark_cell(v, cell, touched);
        const int valid = cell_valid(v, cell);
        const double F = valid ? trilinear_in_cell(v, cell, fr, NULL) : 0.0;
        out.flags |= sample_flags(v, q, valid, F, c);
        if (!valid) { state = 0; continue; }
        if (state == 1 && F <= 0.0) {
            /* bracket (tau_prev, tau]: bisection on the trilinear interpolant */
            double a = tau_prev, b = tau;
            for (int it = 0; it < 64; ++it) {
                const double m = 0.5 * (a + b);
                if (m <= a || m >= b) break;
                double qm[3];
                for (int e = 0; e < 3; ++e) qm[e] = q0[e] + m * dv[e];
                int64_t cm[3];
                double fm[3];
                cell_of(v, qm, cm, fm);
                if (touched) mark_cell(v, cm, touched);
                const double g = trilinear_in_cell(v, cm, fm, NULL);
                if (g > 0.0) a = m; else b = m;
            }
            const double ts = 0.5 * (a + b);
            double qs[3];
            for (int e = 0; e < 3; ++e) qs[e] = q0[e] + ts * dv[e];
            int64_t cs[3];
            double fs[3];
            cell_of(v, qs, cs, fs);
            for (int e = 0; e < 3; ++e) {
                const double fq = fs[e];
                if (fq < c->eps_q || fq > 1.0 - c->eps_q) out.flags |= ORC_RF_FACE;
            }
            out.hit = 1;
            out.tau = ts;
            if (touched) mark_cell(v, cs, touched);
            out.cell_ok = cell_valid(v, cs);
            trilinear_in_cell(v, cs, fs, out.grad);
            if (v->rgba) {
                if (touched_rgb) mark_cell(v, cs, touched_rgb);
                for (int ch = 0; ch < 3; ++ch) {
                    double acc = 0.0;
                    for (int dz = 0; dz < 2; ++dz)
                        for (int dy = 0; dy < 2; ++dy)
                            for (int dx = 0; dx < 2; ++dx) {
                                const double wx = dx ? fs[0] : 1.0 - fs[0];
                                const double wy = dy ? fs[1] : 1.0 - fs[1];
                                const double wz = dz ? fs[2] : 1.0 - fs[2];
                                const size_t vi = vox_index(v, cs[0] + dx, cs[1] + dy, cs[2] + dz);
                                acc += wx * wy * wz * (double)v->rgba[4 * vi + ch];
                            }
                    out.rgb[ch] = acc;
                }
            }
            return out;
        }
        state = (F > 0.0) ? 1 : -1;
        tau_prev = tau;
    }
    return out;
}

static orc_hit march_volume(const orc_volume *v, const double o[3], const double d[3],
                            const orc_config *c)
{
    return march_volume_marking(v, o, d, c, NULL, NULL);
}

/* One pixel: march every volume, keep the nearest hit (exact ties to the
 * lower id), write that pixel's outputs. */
static void raycast_pixel(const orc_volume *vols, const int32_t *ids, int32_t nvol,
                          const orc_intrinsics *K, const double R[9], const double t[3],
                          const orc_config *c, int64_t x, int64_t y, orc_hit *hits,
                          double *depth, double *normal, uint8_t *rgba, double *vertex,
                          int32_t *hit_vol, uint8_t *flags)
{
    const double dc[3] = { ((double)x - K->cx) / K->fx, ((double)y - K->cy) / K->fy, 1.0 };
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = R[3 * a + 0] * dc[0] + R[3 * a + 1] * dc[1] + R[3 * a + 2] * dc[2];
    orc_hit best;
    memset(&best, 0, sizeof(best));
    int32_t best_v = -1;
    uint8_t fl = 0;
    for (int32_t vi = 0; vi < nvol; ++vi) {
        orc_hit hv = march_volume(&vols[vi], t, d, c);
        fl |= hv.flags;
        hits[vi] = hv;
        if (!hv.hit) continue;
        if (best_v < 0 || hv.tau < best.tau || (hv.tau == best.tau && ids[vi] < ids[best_v])) {
            best = hv;
            best_v = vi;
        }
    }
    /* near-ties between volumes matter only where they disagree */
    if (best_v >= 0) {
        for (int32_t vi = 0; vi < nvol; ++vi) {
            if (vi == best_v || !hits[vi].hit) continue;
            if (fabs(hits[vi].tau - best.tau) > 1e-3 * vols[vi].s) continue;
            int differ = hits[vi].cell_ok != best.cell_ok;
            for (int a = 0; a < 3; ++a) {
                if (fabs(hits[vi].grad[a] - best.grad[a]) > 1e-6) differ = 1;
                if (fabs(hits[vi].rgb[a] - best.rgb[a]) > 1e-6) differ = 1;
            }
            if (differ) fl |= ORC_RF_TIE;
        }
    }
    const size_t p = (size_t)y * (size_t)K->width + (size_t)x;
    if (hit_vol) hit_vol[p] = best_v >= 0 ? ids[best_v] : -1;
    if (depth) depth[p] = best_v >= 0 ? best.tau : 0.0;
    double n[3] = {0.0, 0.0, 0.0};
    if (best_v >= 0 && best.cell_ok) {
        const double gn = sqrt(best.grad[0] * best.grad[0] + best.grad[1] * best.grad[1] +
                               best.grad[2] * best.grad[2]);
        if (gn > 0.0) for (int a = 0; a < 3; ++a) n[a] = best.grad[a] / gn;
        if (gn < 1e-3) fl |= ORC_RF_GRAD;
    }
    if (flags) flags[p] = fl;
    if (normal) for (int a = 0; a < 3; ++a) normal[3 * p + a] = n[a];
    if (vertex) for (int a = 0; a < 3; ++a) vertex[3 * p + a] = best_v >= 0 ? t[a] + best.tau * d[a] : 0.0;
    if (rgba) {
        for (int ch = 0; ch < 3; ++ch)
            rgba[4 * p + ch] = (best_v >= 0 && best.cell_ok) ? (uint8_t)floor(best.rgb[ch] + 0.5) : 0;
        rgba[4 * p + 3] = best_v >= 0 ? 255 : 0;
    }
}

/* Raycast a view of all given volumes into one map (shortest distance wins).
 * Outputs (each may be NULL): depth[h*w] (0 = no hit), normal[h*w*3],
 * rgba[h*w*4], vertex[h*w*3], hit_vol[h*w] (-1 = no hit), flags[h*w].
 * ids gives each volume's id for tie-breaking (lower id wins). */
ORC_EXPORT void orc_raycast(const orc_volume *vols, const int32_t *ids, int32_t nvol,
                            const orc_intrinsics *K, const double T[16], const orc_config *c,
                            double *depth, double *normal, uint8_t *rgba, double *vertex,
                            int32_t *hit_vol, uint8_t *flags)
{
    double R[9], t[3];
    pose_split(T, R, t);
    const int64_t W = K->width, H = K->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t y = 0; y < H; ++y) {
        orc_hit hits[nvol > 0 ? nvol : 1];
        for (int64_t x = 0; x < W; ++x)
            raycast_pixel(vols, ids, nvol, K, R, t, c, x, y, hits, depth, normal, rgba, vertex,
                          hit_vol, flags);
    }
}

/* The same for a list of pixels (linear indices y * width + x); outputs are
 * full-size maps of which only the listed pixels are written. */
ORC_EXPORT void orc_raycast_pixels(const orc_volume *vols, const int32_t *ids, int32_t nvol,
                                   const orc_intrinsics *K, const double T[16], const orc_config *c,
                                   const int64_t *pix, int64_t npix, double *depth, double *normal,
                                   uint8_t *rgba, double *vertex, int32_t *hit_vol, uint8_t *flags)
{
    double R[9], t[3];
    pose_split(T, R, t);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < npix; ++j) {
        orc_hit hits[nvol > 0 ? nvol : 1];
        raycast_pixel(vols, ids, nvol, K, R, t, c, pix[j] % K->width, pix[j] / K->width, hits,
                      depth, normal, rgba, vertex, hit_vol, flags);
    }
}

/* Memory footprint of a raycast (the bytes a dense march must read): every
 * pixel (or the listed ones) is marched through every volume as orc_raycast
 * does, and counts[2 v] receives the number of distinct voxels of volume v
 * whose (F, W) the march reads (the 2x2x2 neighbourhoods of its samples and
 * bisection midpoints), counts[2 v + 1] the number of distinct voxels whose
 * colour the hits read.  Returns 0, or -1 when a bitmap cannot be allocated. */
ORC_EXPORT int orc_raycast_footprint(const orc_volume *vols, int32_t nvol, const orc_intrinsics *K,
                                     const double T[16], const orc_config *c, const int64_t *pix,
                                     int64_t npix, int64_t *counts)
{
    double R[9], t[3];
    pose_split(T, R, t);
    uint64_t **bits = (uint64_t **)calloc((size_t)(nvol > 0 ? 2 * nvol : 1), sizeof(uint64_t *));
    if (!bits) return -1;
    int ok = 1;
    for (int32_t vi = 0; vi < nvol && ok; ++vi) {
        const size_t n = (size_t)vols[vi].r[0] * vols[vi].r[1] * vols[vi].r[2];
        bits[2 * vi] = (uint64_t *)calloc((n + 63) / 64, sizeof(uint64_t));
        bits[2 * vi + 1] = (uint64_t *)calloc((n + 63) / 64, sizeof(uint64_t));
        ok = bits[2 * vi] && bits[2 * vi + 1];
    }
    if (ok) {
        const int64_t total = pix ? npix : (int64_t)K->width * K->height;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t j = 0; j < total; ++j) {
            const int64_t p = pix ? pix[j] : j;
            const double x = (double)(p % K->width), y = (double)(p / K->width);
            const double dc[3] = { (x - K->cx) / K->fx, (y - K->cy) / K->fy, 1.0 };
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = R[3 * a + 0] * dc[0] + R[3 * a + 1] * dc[1] + R[3 * a + 2] * dc[2];
            for (int32_t vi = 0; vi < nvol; ++vi)
                march_volume_marking(&vols[vi], t, d, c, bits[2 * vi], bits[2 * vi + 1]);
        }
        for (int32_t vi = 0; vi < nvol; ++vi) {
            const size_t n = (size_t)vols[vi].r[0] * vols[vi].r[1] * vols[vi].r[2];
            for (int k = 0; k < 2; ++k) {
                int64_t cnt = 0;
                for (size_t w = 0; w < (n + 63) / 64; ++w) cnt += __builtin_popcountll(bits[2 * vi + k][w]);
                counts[2 * vi + k] = cnt;
            }
        }
    }
    for (int32_t vi = 0; vi < 2 * nvol; ++vi) free(bits[vi]);
    free(bits);
    return ok ? 0 : -1;
}

/* Trilinear value and validity at one point q (this volume's voxel
 * coordinates) -- exposed for tests. */
ORC_EXPORT double orc_sample(const orc_volume *v, const double q[3], int32_t *valid)
{
    int64_t cell[3];
    double fr[3];
    const double g[3] = { q[0] + v->h[0], q[1] + v->h[1], q[2] + v->h[2] };
    cell_of(v, g, cell, fr);
    if (valid) *valid = cell_valid(v, cell);
    return trilinear_in_cell(v, cell, fr, NULL);
}

/* ------------------------------------------------------------------------ */
/* Gradients of the raycast (not in the paper: the differentiable form of   */
/* the raycast used for pose refinement).                                   */
/*                                                                          */
/* The pose is perturbed on the left, T(xi) = exp(xi^) T with              */
/* xi = (rho, phi) in the world frame, so a point x of the ray moves by     */
/* dx/dxi = [ I | -[x]_x ].  The hit tau* solves F(t + tau d) = 0; with the  */
/* analytic trilinear gradient g at x* and the hit cell's weights w_j:      */
/*   dtau/dxi = -(g, x* x g) / (g.d),   dtau/dF_j = -w_j / (g.d),           */
/*   d(x*)/dxi  = [ I | -[x*]_x ] + d dtau/dxi,                               */
/*   C(x) = sum_j w_j(x) c_j / 255 (unrounded colour of the hit cell),      */
/*   dC/dxi = J_C d(x*)/dxi,   dC/dF_j = J_C d dtau/dF_j  (colour voxels are  */
/* constants).  Pixels without a hit, with an unobserved corner in the hit  */
/* cell, at grazing incidence (|g.d| <= 1e-3 |g||d|) or within eps_q of a   */
/* cell face (where the interpolant's gradient jumps) are excluded.         */
/* ------------------------------------------------------------------------ */
enum { ORC_GX_NOHIT = 1, ORC_GX_CELL = 2, ORC_GX_FACE = 4, ORC_GX_GRAZE = 8 };

/* Gradients of one pixel's hit (the body of orc_raycast_grad). */
static void grad_pixel(const orc_volume *vols, const int32_t *ids, int32_t nvol, const orc_intrinsics *K,
                       const double R[9], const double t[3], const orc_config *c, int64_t x, int64_t y,
                       double *depth, const double *grad_depth, const double *grad_rgb, double *grad_pose,
                       double *jac_tau, double *jac_rgb, double **grad_F, uint8_t *excluded)
{
    const int64_t W = K->width;
    const size_t p = (size_t)y * (size_t)W + (size_t)x;
    if (jac_tau) for (int k = 0; k < 6; ++k) jac_tau[6 * p + k] = 0.0;
    if (jac_rgb) for (int k = 0; k < 18; ++k) jac_rgb[18 * p + k] = 0.0;
    const double dc[3] = { ((double)x - K->cx) / K->fx, ((double)y - K->cy) / K->fy, 1.0 };
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = R[3 * a + 0] * dc[0] + R[3 * a + 1] * dc[1] + R[3 * a + 2] * dc[2];
    orc_hit best;
    memset(&best, 0, sizeof(best));
    int32_t best_v = -1;
    for (int32_t vi = 0; vi < nvol; ++vi) {
        orc_hit hv = march_volume(&vols[vi], t, d, c);
        if (!hv.hit) continue;
        if (best_v < 0 || hv.tau < best.tau || (hv.tau == best.tau && ids[vi] < ids[best_v])) {
            best = hv;
            best_v = vi;
        }
    }
    uint8_t ex = 0;
    if (depth) depth[p] = best_v >= 0 ? best.tau : 0.0;
    if (best_v < 0) {
        if (excluded) excluded[p] = ORC_GX_NOHIT;
        return;
    }
    const orc_volume *v = &vols[best_v];
    const double s = v->s, tau = best.tau;
    double q[3], xs[3];
    for (int a = 0; a < 3; ++a) {
        q[a] = t[a] / s + tau * (d[a] / s);
        xs[a] = t[a] + tau * d[a];
    }
    int64_t cell[3];
    double fr[3];
    cell_of(v, q, cell, fr);
    if (!cell_valid(v, cell)) ex |= ORC_GX_CELL;
    for (int a = 0; a < 3; ++a)
        if (fr[a] < c->eps_q || fr[a] > 1.0 - c->eps_q) ex |= ORC_GX_FACE;
    /* corner values, weights and weight gradients (per metre) */
    double wj[8], gw[8][3], Fj[8], cj[8][3];
    double g[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const double wx = dx ? fr[0] : 1.0 - fr[0];
        const double wy = dy ? fr[1] : 1.0 - fr[1];
        const double wz = dz ? fr[2] : 1.0 - fr[2];
        wj[k] = wx * wy * wz;
        gw[k][0] = (dx ? 1.0 : -1.0) * wy * wz / s;
        gw[k][1] = wx * (dy ? 1.0 : -1.0) * wz / s;
        gw[k][2] = wx * wy * (dz ? 1.0 : -1.0) / s;
        const size_t vi = vox_index(v, cell[0] + dx, cell[1] + dy, cell[2] + dz);
        Fj[k] = v->F[vi];
        for (int ch = 0; ch < 3; ++ch) cj[k][ch] = v->rgba ? v->rgba[4 * vi + ch] / 255.0 : 0.0;
        for (int a = 0; a < 3; ++a) g[a] += Fj[k] * gw[k][a];
    }
    const double gd = g[0] * d[0] + g[1] * d[1] + g[2] * d[2];
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(fabs(gd) > 1e-3 * gn * dn)) ex |= ORC_GX_GRAZE;
    if (excluded) excluded[p] = ex;
    if (ex) return;
    /* dtau/dxi */
    double jt[6];
    const double xg[3] = { xs[1] * g[2] - xs[2] * g[1], xs[2] * g[0] - xs[0] * g[2],
                           xs[0] * g[1] - xs[1] * g[0] };
    for (int a = 0; a < 3; ++a) {
        jt[a] = -g[a] / gd;
        jt[3 + a] = -xg[a] / gd;
    }
    /* d(x*)/dxi = [I | -[x*]_x] + d jt^T */
    double dxdxi[3][6];
    const double mX[3][3] = { {0.0, xs[2], -xs[1]}, {-xs[2], 0.0, xs[0]}, {xs[1], -xs[0], 0.0} };
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 6; ++b)
            dxdxi[a][b] = (b < 3 ? (a == b ? 1.0 : 0.0) : mX[a][b - 3]) + d[a] * jt[b];
    /* colour Jacobian J_C (3x3, per metre) and dC/dxi */
    double JC[3][3] = {{0.0}};
    for (int k = 0; k < 8; ++k)
        for (int ch = 0; ch < 3; ++ch)
            for (int a = 0; a < 3; ++a) JC[ch][a] += cj[k][ch] * gw[k][a];
    double jc[3][6];
    for (int ch = 0; ch < 3; ++ch)
        for (int b = 0; b < 6; ++b) {
            jc[ch][b] = 0.0;
            for (int a = 0; a < 3; ++a) jc[ch][b] += JC[ch][a] * dxdxi[a][b];
        }
    if (jac_tau) for (int b = 0; b < 6; ++b) jac_tau[6 * p + b] = jt[b];
    if (jac_rgb)
        for (int ch = 0; ch < 3; ++ch)
            for (int b = 0; b < 6; ++b) jac_rgb[18 * p + 6 * ch + b] = jc[ch][b];
    const double gdep = grad_depth ? grad_depth[p] : 0.0;
    double gc[3] = {0.0, 0.0, 0.0};
    if (grad_rgb) for (int ch = 0; ch < 3; ++ch) gc[ch] = grad_rgb[3 * p + ch];
    if (grad_pose)
        for (int b = 0; b < 6; ++b) {
            double acc = gdep * jt[b];
            for (int ch = 0; ch < 3; ++ch) acc += gc[ch] * jc[ch][b];
            grad_pose[b] += acc;
        }
    if (grad_F && grad_F[best_v]) {
        /* dtau/dF_j = -w_j / gd; dC/dF_j = J_C d dtau/dF_j */
        double jcd = 0.0;
        for (int ch = 0; ch < 3; ++ch)
            jcd += gc[ch] * (JC[ch][0] * d[0] + JC[ch][1] * d[1] + JC[ch][2] * d[2]);
        const double coef = -(gdep + jcd) / gd;
        for (int k = 0; k < 8; ++k) {
            const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
            grad_F[best_v][vox_index(v, cell[0] + dx, cell[1] + dy, cell[2] + dz)] += coef * wj[k];
        }
    }
}

ORC_EXPORT void orc_raycast_grad(const orc_volume *vols, const int32_t *ids, int32_t nvol,
                                 const orc_intrinsics *K, const double T[16], const orc_config *c,
                                 double *depth, const double *grad_depth, const double *grad_rgb,
                                 double *grad_pose, double *jac_tau, double *jac_rgb,
                                 double **grad_F, uint8_t *excluded)
{
    double R[9], t[3];
    pose_split(T, R, t);
    const int64_t W = K->width, H = K->height;
    if (grad_pose) for (int k = 0; k < 6; ++k) grad_pose[k] = 0.0;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x)
            grad_pixel(vols, ids, nvol, K, R, t, c, x, y, depth, grad_depth, grad_rgb, grad_pose, jac_tau,
                       jac_rgb, grad_F, excluded);
}

/* The same for a list of pixels (linear indices y * width + x, in order);
 * per-pixel outputs are full-size maps of which only the listed pixels are
 * written, and grad_pose / grad_F sum over the listed pixels only. */
ORC_EXPORT void orc_raycast_grad_pixels(const orc_volume *vols, const int32_t *ids, int32_t nvol,
                                        const orc_intrinsics *K, const double T[16], const orc_config *c,
                                        const int64_t *pix, int64_t npix, double *depth,
                                        const double *grad_depth, const double *grad_rgb, double *grad_pose,
                                        double *jac_tau, double *jac_rgb, double **grad_F, uint8_t *excluded)
{
    double R[9], t[3];
    pose_split(T, R, t);
    if (grad_pose) for (int k = 0; k < 6; ++k) grad_pose[k] = 0.0;
    for (int64_t j = 0; j < npix; ++j)
        grad_pixel(vols, ids, nvol, K, R, t, c, pix[j] % K->width, pix[j] / K->width, depth, grad_depth,
                   grad_rgb, grad_pose, jac_tau, jac_rgb, grad_F, excluded);
}

/* ------------------------------------------------------------------------
 * Placement lattice (Sec. Dynamic Mapping for SLAM).  For every pixel (x, y)
 * with a valid depth D the ray endpoint is e = T (D K^-1 [x, y, 1]^T) in
 * world metres: with xn = (x - cx) / fx and yn = (y - cy) / fy the camera
 * point is (D xn, D yn, D) and e_a = R_a0 (D xn) + R_a1 (D yn) + R_a2 D + t_a,
 * summed left to right.  Its lattice cell is l_a = floor(e_a / cell_m), with
 * cell_m = (d_v - 2) * pitch, the spacing of the volume origins
 * h_t = k (d_v - 2).  (The paper's printed endpoint formula is garbled; this
 * is the back-projection it describes.)  valid[p] = 0 where the depth is
 * not valid (not > 0, or outside [z_min, z_max]); cells then are 0.
 * ------------------------------------------------------------------------ */
ORC_EXPORT void orc_endpoint_cells(const float *depth, const orc_intrinsics *K, const double T[16],
                                   double z_min, double z_max, double cell_m, int64_t *cells,
                                   uint8_t *valid)
{
    const int W = K->width, H = K->height;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const double D = (double)depth[p];
            cells[3 * p] = cells[3 * p + 1] = cells[3 * p + 2] = 0;
            valid[p] = 0;
            if (!(D > 0.0) || D < z_min || D > z_max) continue;
            const double xn = ((double)x - K->cx) / K->fx;
            const double yn = ((double)y - K->cy) / K->fy;
            const double pc[3] = {D * xn, D * yn, D};
            for (int a = 0; a < 3; ++a) {
                const double e = T[4 * a] * pc[0] + T[4 * a + 1] * pc[1] + T[4 * a + 2] * pc[2] + T[4 * a + 3];
                cells[3 * p + a] = (int64_t)floor(e / cell_m);
            }
            valid[p] = 1;
        }
}

/* ------------------------------------------------------------------------
 * Surface points of a volume (Sec. Insertion and Removal: a volume leaves the
 * map as a point cloud; Table 1 counts such points).  For every voxel i and
 * axis a with i + e_a inside the volume, both observed (W > 0) and on
 * different sides of the surface, (F_i > 0) != (F_{i+e_a} > 0): one point at
 * the zero of the linear interpolation along the edge, t = F_i / (F_i -
 * F_{i+e_a}), p = (h + i + t e_a) s, coloured c_i + t (c_{i+e_a} - c_i) per
 * channel, rounded half up.  Points come by increasing edge id
 * 3 * lin(i) + a (lin: x fastest).  Returns the number of points; writes at
 * most cap of them (any output may be NULL).
 * ------------------------------------------------------------------------ */
ORC_EXPORT int64_t orc_extract_points(const orc_volume *v, double *xyz, uint8_t *rgb, int64_t *edge,
                                      int64_t cap)
{
    const int64_t rx = v->r[0], ry = v->r[1], rz = v->r[2];
    int64_t n = 0;
    for (int64_t z = 0; z < rz; ++z)
        for (int64_t y = 0; y < ry; ++y)
            for (int64_t x = 0; x < rx; ++x) {
                const int64_t i = (z * ry + y) * rx + x;
                if (!(v->W[i] > 0.0)) continue;
                for (int a = 0; a < 3; ++a) {
                    const int64_t q[3] = {x + (a == 0), y + (a == 1), z + (a == 2)};
                    if (q[0] >= rx || q[1] >= ry || q[2] >= rz) continue;
                    const int64_t j = (q[2] * ry + q[1]) * rx + q[0];
                    if (!(v->W[j] > 0.0)) continue;
                    if ((v->F[i] > 0.0) == (v->F[j] > 0.0)) continue;
                    const double t = v->F[i] / (v->F[i] - v->F[j]);
                    if (n < cap) {
                        const int64_t p[3] = {x, y, z};
                        if (xyz)
                            for (int b = 0; b < 3; ++b)
                                xyz[3 * n + b] = ((double)(v->h[b] + p[b]) + (b == a ? t : 0.0)) * v->s;
                        if (rgb)
                            for (int ch = 0; ch < 3; ++ch) {
                                const double c0 = v->rgba ? v->rgba[4 * i + ch] : 0.0;
                                const double c1 = v->rgba ? v->rgba[4 * j + ch] : 0.0;
                                const double cv = floor(c0 + t * (c1 - c0) + 0.5);
                                rgb[3 * n + ch] = (uint8_t)(cv > 255.0 ? 255.0 : cv);
                            }
                        if (edge) edge[n] = 3 * i + a;
                    }
                    ++n;
                }
            }
    return n;
}

/* ------------------------------------------------------------------------
 * Depth-map conversion (Sec. Depth Map Conversion): v = K^-1 [x, y, 1]^T D
 * for valid depths (> 0, inside [z_min, z_max]); n = (v(x+1, y) - v(x, y)) x
 * (v(x, y+1) - v(x, y)) where the three depths are valid, normalised and
 * turned to face the camera (n . v < 0; the paper's cross product of the
 * two image-axis differences points away from the camera).  With T non-NULL
 * both go to the world frame (R v + t, R n).  Invalid entries are 0.
 * ------------------------------------------------------------------------ */
static int depth_ok(double D, double z_min, double z_max)
{
    return D > 0.0 && D >= z_min && D <= z_max;
}

ORC_EXPORT void orc_depth_maps(const float *depth, const orc_intrinsics *K, const double *T, double z_min,
                               double z_max, double *vertex, double *normal)
{
    const int W = K->width, H = K->height;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            double v[3] = {0, 0, 0}, n[3] = {0, 0, 0};
            const double D = depth[p];
            const int ok = depth_ok(D, z_min, z_max);
            if (ok) {
                v[0] = (x - K->cx) / K->fx * D;
                v[1] = (y - K->cy) / K->fy * D;
                v[2] = D;
                if (x + 1 < W && y + 1 < H && depth_ok(depth[p + 1], z_min, z_max) &&
                    depth_ok(depth[p + W], z_min, z_max)) {
                    const double Dx = depth[p + 1], Dy = depth[p + W];
                    const double a[3] = {(x + 1 - K->cx) / K->fx * Dx - v[0], (y - K->cy) / K->fy * Dx - v[1],
                                         Dx - v[2]};
                    const double b[3] = {(x - K->cx) / K->fx * Dy - v[0], (y + 1 - K->cy) / K->fy * Dy - v[1],
                                         Dy - v[2]};
                    double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
                    const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
                    if (len > 0.0) {
                        const double sg = (c[0] * v[0] + c[1] * v[1] + c[2] * v[2] > 0.0) ? -1.0 : 1.0;
                        for (int k = 0; k < 3; ++k) n[k] = sg * c[k] / len;
                    }
                }
            }
            for (int a = 0; a < 3; ++a) {
                double vo = v[a], no = n[a];
                if (T && ok) {
                    vo = T[4 * a] * v[0] + T[4 * a + 1] * v[1] + T[4 * a + 2] * v[2] + T[4 * a + 3];
                    no = T[4 * a] * n[0] + T[4 * a + 1] * n[1] + T[4 * a + 2] * n[2];
                }
                vertex[3 * p + a] = ok ? vo : 0.0;
                normal[3 * p + a] = ok ? no : 0.0;
            }
        }
}

/* ------------------------------------------------------------------------
 * One point-to-plane ICP linearisation with projective data association
 * (Sec. Camera Tracking, the KinectFusion tracker it cites).  For each pixel
 * of the current frame with a normal (camera-frame maps v, n): v_g = R v + t,
 * n_g = R n with T_est = [R | t]; q = T_model^-1 v_g; the nearest model pixel
 * (floor(fx q_x / q_z + cx + 1/2), same for y) if q_z > 0 and it is inside
 * the image; the model vertex V and normal N there (|N|^2 > 1/4, i.e. not a
 * miss); association when |v_g - V|^2 <= dist^2 and n_g . N >= cos_min.
 * r = N . (V - v_g), J = [N, v_g x N]; sums of J^T J (A, row-major 6x6),
 * J^T r (b), r^2 and the count.  flags[p] = 1 for pixels whose association
 * decision lies within a small margin of a threshold (another evaluation in
 * lower precision may decide differently); absA / absb / abse receive the
 * sums of |term| over those flagged pixels.
 * ------------------------------------------------------------------------ */
ORC_EXPORT void orc_icp_system(const double *vertex, const double *normal, const orc_intrinsics *K,
                               const double *T_est, const float *mvertex, const float *mnormal,
                               const double *T_model, double dist, double cos_min, double *A, double *b,
                               double *err, int64_t *count, uint8_t *flags, double *absA, double *absb,
                               double *abse)
{
    const int W = K->width, H = K->height;
    const double eps_px = 2e-3, eps_rel = 1e-4, eps_cos = 1e-3;
    for (int k = 0; k < 36; ++k) A[k] = absA[k] = 0.0;
    for (int k = 0; k < 6; ++k) b[k] = absb[k] = 0.0;
    *err = 0.0;
    abse[0] = abse[1] = 0.0;
    *count = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            flags[p] = 0;
            const double *n = normal + 3 * p, *v = vertex + 3 * p;
            if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) continue;
            double vg[3], ng[3], d[3], q[3];
            for (int a = 0; a < 3; ++a) {
                vg[a] = T_est[4 * a] * v[0] + T_est[4 * a + 1] * v[1] + T_est[4 * a + 2] * v[2] + T_est[4 * a + 3];
                ng[a] = T_est[4 * a] * n[0] + T_est[4 * a + 1] * n[1] + T_est[4 * a + 2] * n[2];
            }
            for (int a = 0; a < 3; ++a) d[a] = vg[a] - T_model[4 * a + 3];
            for (int a = 0; a < 3; ++a) q[a] = T_model[a] * d[0] + T_model[4 + a] * d[1] + T_model[8 + a] * d[2];
            if (!(q[2] > 0.0)) continue;
            const double u = K->fx * q[0] / q[2] + K->cx, w = K->fy * q[1] / q[2] + K->cy;
            const double fu = u + 0.5 - floor(u + 0.5), fw = w + 0.5 - floor(w + 0.5);
            int marginal = fu < eps_px || fu > 1.0 - eps_px || fw < eps_px || fw > 1.0 - eps_px;
            const int64_t ui = (int64_t)floor(u + 0.5), wi = (int64_t)floor(w + 0.5);
            if (ui < 0 || wi < 0 || ui >= W || wi >= H) {
                if (marginal) flags[p] = 1;
                continue;
            }
            const size_t m = (size_t)wi * W + ui;
            const double N[3] = {mnormal[3 * m], mnormal[3 * m + 1], mnormal[3 * m + 2]};
            if (!(N[0] * N[0] + N[1] * N[1] + N[2] * N[2] > 0.25)) {
                if (marginal) flags[p] = 1;
                continue;
            }
            const double V[3] = {mvertex[3 * m], mvertex[3 * m + 1], mvertex[3 * m + 2]};
            const double e[3] = {V[0] - vg[0], V[1] - vg[1], V[2] - vg[2]};
            const double d2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
            const double cs = ng[0] * N[0] + ng[1] * N[1] + ng[2] * N[2];
            marginal |= fabs(d2 - dist * dist) < eps_rel * dist * dist || fabs(cs - cos_min) < eps_cos;
            if (marginal) flags[p] = 1;
            if (!(d2 <= dist * dist) || !(cs >= cos_min)) continue;
            const double r = N[0] * e[0] + N[1] * e[1] + N[2] * e[2];
            const double J[6] = {N[0], N[1], N[2], vg[1] * N[2] - vg[2] * N[1], vg[2] * N[0] - vg[0] * N[2],
                                 vg[0] * N[1] - vg[1] * N[0]};
            for (int i = 0; i < 6; ++i) {
                for (int j = 0; j < 6; ++j) {
                    A[6 * i + j] += J[i] * J[j];
                    if (marginal) absA[6 * i + j] += fabs(J[i] * J[j]);
                }
                b[i] += J[i] * r;
                if (marginal) absb[i] += fabs(J[i] * r);
            }
            *err += r * r;
            *count += 1;
            if (marginal) {
                abse[0] += r * r;
                abse[1] += 1.0;
            }
        }
}

/* Threads an OpenMP loop of this library uses (1 without OpenMP). */
ORC_EXPORT int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the threads of this library's OpenMP loops (n >= 1). */
ORC_EXPORT void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
