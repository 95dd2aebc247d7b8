// mv_raycast.cu -- per-pixel raycast of all resident volumes (sm_103a).
//
// Sec. Raycasting / Algorithm 1 (second loop) of Salvato, Finman, Leonard,
// arXiv 1511.07106: each pixel's ray is marched through each volume, the
// zero crossing of the trilinearly interpolated TSDF gives the vertex, the
// TSDF derivative there gives the normal, and all volumes write one map where
// the shortest ray distance wins.
//
// March semantics (identical to the FP64 oracle): samples lie on the global
// grid tau_k = k * Delta, Delta = step * s / |d|, positions are taken in
// global voxel coordinates (the paper's t_r; volume coordinates t_r - h_t),
// a sample is valid when the 8 corners of its cell are observed (W > 0), and
// the first pair of consecutive valid samples going from F > 0 to F <= 0
// brackets the surface, refined by bisection and a final secant step.
//
// B300 design: one thread per pixel, 8x4-pixel warp tiles for gather
// locality, every volume of the view in one launch with the nearest hit kept
// in registers; each CTA first keeps only the volumes its pixel rectangle can
// hit.  Space that cannot hold a surface crossing is crossed by a 3D DDA over
// 8^3-voxel cell bricks and 32^3-voxel super bricks using exact per-brick
// summaries (see march_volume): a shortcut, not an approximation.  The
// bisection keeps the corners of its current cell in registers.
#include <float.h>
#include <limits.h>

#include "mv_internal.cuh"

namespace mv {

struct RayOut {
    float *depth;
    float *normal;
    uint32_t *rgba;
    float *vertex;
    int *vol_id;
};

template <int FMT, typename Off>
__device__ __forceinline__ void load_fw(const VolDev &v, Off off, float &F, float &W)
{
    if (FMT == MV_TSDF_F32) {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(v.fw) + off);
        F = q.x;
        W = q.y;
    } else {
        const uint32_t q = __ldg(reinterpret_cast<const uint32_t *>(v.fw) + off);
        if (FMT == MV_TSDF_F16) decode_f16(q, F, W); else decode_i16(q, F, W);
    }
}

// Brick-layout strides of one volume, hoisted out of the march.  Off is
// uint32_t for volumes of fewer than 2^32 voxels (cheaper address math), else
// long long.
template <typename Off>
struct Geo {
    Off nb0, nb01;  // bricks per row, per slice
    Off oy, oz;     // element step to the +y / +z neighbour across a brick face
    int nby;
};

template <typename Off>
__device__ __forceinline__ Geo<Off> make_geo(const VolDev &v)
{
    Geo<Off> g;
    g.nb0 = (Off)v.nb[0];
    g.nb01 = (Off)v.nb[0] * (Off)v.nb[1];
    g.oy = g.nb0 * (Off)kBrickVox - (Off)56;
    g.oz = g.nb01 * (Off)kBrickVox - (Off)448;
    g.nby = v.nb[1];
    return g;
}

// Offsets of the 8 corners of the cell with lower corner (x, y, z).
template <typename Off>
struct Corners {
    Off base, ox, oy, oz;
};

template <typename Off>
__device__ __forceinline__ Corners<Off> cell_corners(const Geo<Off> &g, int x, int y, int z)
{
    Corners<Off> c;
    const Off b = (Off)(z >> 3) * g.nb01 + (Off)(y >> 3) * g.nb0 + (Off)(x >> 3);
    c.base = b * (Off)kBrickVox + (Off)(((z & 7) << 6) | ((y & 7) << 3) | (x & 7));
    c.ox = ((x & 7) == 7) ? (Off)(kBrickVox - 7) : (Off)1;
    c.oy = ((y & 7) == 7) ? g.oy : (Off)8;
    c.oz = ((z & 7) == 7) ? g.oz : (Off)64;
    return c;
}

// Trilinear F in a cell; valid = all 8 corners observed.
template <int FMT, typename Off>
__device__ __forceinline__ float trilinear(const VolDev &v, const Corners<Off> &c, float fx, float fy,
                                           float fz, bool &valid)
{
    float F[8], W[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const Off off = c.base + ((k & 1) ? c.ox : (Off)0) + ((k & 2) ? c.oy : (Off)0) + ((k & 4) ? c.oz : (Off)0);
        load_fw<FMT>(v, off, F[k], W[k]);
    }
    valid = (W[0] > 0.f) & (W[1] > 0.f) & (W[2] > 0.f) & (W[3] > 0.f) & (W[4] > 0.f) &
            (W[5] > 0.f) & (W[6] > 0.f) & (W[7] > 0.f);
    const float x00 = fmaf(fx, F[1] - F[0], F[0]);
    const float x10 = fmaf(fx, F[3] - F[2], F[2]);
    const float x01 = fmaf(fx, F[5] - F[4], F[4]);
    const float x11 = fmaf(fx, F[7] - F[6], F[6]);
    const float y0 = fmaf(fy, x10 - x00, x00);
    const float y1 = fmaf(fy, x11 - x01, x01);
    return fmaf(fz, y1 - y0, y0);
}

// Per-volume ray state in this volume's global voxel units, relative to the
// camera's lattice point cam_int: sample k sits at rr(k) = cam_frac + k * dq.
struct VolRay {
    float fr[3];   // cam_frac
    float dq[3];   // grid step in voxels
    int oi[3];     // cam_int - h_t (local index of the camera's lattice point)
};

// Cell (local, clamped) and fractions of the point rr (camera-relative).
// Cell only (the march decides most samples from the cell's masks).
__device__ __forceinline__ void locate_cell(const VolDev &v, const VolRay &vr, const float rr[3], int cell[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) cell[a] = max(0, min(v.r[a] - 2, __float2int_rd(rr[a]) + vr.oi[a]));
}

__device__ __forceinline__ void locate(const VolDev &v, const VolRay &vr, const float rr[3],
                                       int cell[3], float f[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(rr[a]);
        int c = (int)fl + vr.oi[a];
        c = max(0, min(v.r[a] - 2, c));
        cell[a] = c;
        f[a] = rr[a] - (float)(c - vr.oi[a]);
    }
}

template <int FMT, typename Off>
__device__ __forceinline__ float eval_at(const VolDev &v, const Geo<Off> &g, const VolRay &vr, float k,
                                         bool &valid)
{
    float rr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) rr[a] = fmaf(k, vr.dq[a], vr.fr[a]);
    int cell[3];
    float f[3];
    locate(v, vr, rr, cell, f);
    const Corners<Off> c = cell_corners(g, cell[0], cell[1], cell[2]);
    return trilinear<FMT>(v, c, f[0], f[1], f[2], valid);
}

struct RayCount {
    unsigned samples, skips, hits;
};

// Nearest hit so far: ray distance, volume id and table slot, and the sample
// parameter of the refined root in that volume's grid (the shading happens
// once, after every volume has been marched).
struct Hit {
    float tau;
    int id;
    int slot;
    float ks;
};

// Normal and colour of a hit.
struct Shade {
    float n[3];
    uint32_t rgba;
};

// Gradient (normal) and colour in the hit cell.
template <int FMT, typename Off>
__device__ __forceinline__ void shade(const VolDev &v, const Geo<Off> &geo, const VolRay &vr, float ks,
                                      Shade &h)
{
    float rr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) rr[a] = fmaf(ks, vr.dq[a], vr.fr[a]);
    int cell[3];
    float f[3];
    locate(v, vr, rr, cell, f);
    const Corners<Off> c = cell_corners(geo, cell[0], cell[1], cell[2]);
    float F[8], W[8];
    uint32_t col[8];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const Off off = c.base + ((k & 1) ? c.ox : (Off)0) + ((k & 2) ? c.oy : (Off)0) + ((k & 4) ? c.oz : (Off)0);
        load_fw<FMT>(v, off, F[k], W[k]);
        col[k] = __ldg(v.rgba + off);
        ok &= W[k] > 0.f;
    }
    h.n[0] = h.n[1] = h.n[2] = 0.f;
    h.rgba = 0xFF000000u;
    if (!ok) return;
    const float x = f[0], y = f[1], z = f[2];
    float g[3] = {0.f, 0.f, 0.f};
    float rgb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float wx = (k & 1) ? x : 1.f - x;
        const float wy = (k & 2) ? y : 1.f - y;
        const float wz = (k & 4) ? z : 1.f - z;
        g[0] += ((k & 1) ? 1.f : -1.f) * wy * wz * F[k];
        g[1] += wx * ((k & 2) ? 1.f : -1.f) * wz * F[k];
        g[2] += wx * wy * ((k & 4) ? 1.f : -1.f) * F[k];
        const float w = wx * wy * wz;
        rgb[0] += w * (float)(col[k] & 0xFFu);
        rgb[1] += w * (float)((col[k] >> 8) & 0xFFu);
        rgb[2] += w * (float)((col[k] >> 16) & 0xFFu);
    }
    const float gn2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (gn2 > 0.f) {
        const float inv = rsqrtf(gn2);
        h.n[0] = g[0] * inv;
        h.n[1] = g[1] * inv;
        h.n[2] = g[2] * inv;
    }
    uint32_t out = 0xFF000000u;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const int cv = min(255, max(0, (int)floorf(rgb[ch] + 0.5f)));
        out |= (uint32_t)cv << (8 * ch);
    }
    h.rgba = out;
}

// DDA set-up along one axis: parameter (in samples) of the first brick face
// crossed from L, spacing of the faces, step direction, and the domain end
// (the last voxel plane less m) for positive directions.  Products with the
// rounded reciprocal of dq instead of quotients: a few ulp of the parameters,
// far inside the margin m of the landing.
__device__ __forceinline__ void dda_axis(float L, float dq, int b0, int r, float m, float &tmax,
                                         float &tdel, int &step, float &tdom)
{
    const float rq = __frcp_rn(dq);
    if (dq > 0.f) {
        tmax = ((float)((b0 + 1) * kBrick) - L) * rq;
        tdel = (float)kBrick * rq;
        step = 1;
        tdom = fminf(tdom, ((float)(r - 1) - m - L) * rq);
    } else if (dq < 0.f) {
        tmax = ((float)(b0 * kBrick) - L) * rq;
        tdel = -(float)kBrick * rq;
        step = -1;
    } else {
        tmax = 3.0e38f;
        tdel = 3.0e38f;
        step = 0;
    }
}

// Word of the super brick holding cell brick (bx, by, bz); volumes without
// super bricks read as "not empty".
__device__ __forceinline__ unsigned super_word(const VolDev &v, int bx, int by, int bz)
{
    if (!v.sup) return 1u;
    const unsigned i = (((unsigned)bz >> 2) * (unsigned)v.nsb[1] + ((unsigned)by >> 2)) * (unsigned)v.nsb[0] +
                       ((unsigned)bx >> 2);
    return __ldg(v.sup + i);
}

// Brick boundaries along one axis between brick b and the face, in the step
// direction, of the block of super bricks within Chebyshev distance `reach`
// of b's super brick, clipped to the grid of nb bricks.
__device__ __forceinline__ int inner_faces(int b, int step, int reach, int nb)
{
    return step > 0 ? min(3 - (b & 3) + 4 * reach, nb - 1 - b) : (step < 0 ? min((b & 3) + 4 * reach, b) : 0);
}

// Brick boundaries along one axis crossed by parameter texit (next boundary
// at tmax, spacing tdel = 1 / rdel), at most n.  Rounded down near a
// boundary: the walk then visits a brick the ray only grazes (an earlier
// stop), never skips one.
__device__ __forceinline__ int faces_crossed(float tmax, float rdel, float texit, int n)
{
    if (!(tmax <= texit)) return 0;
    return min(n, (int)floorf(fmaf(texit - tmax, rdel, -1e-4f)) + 1);
}

// 3D DDA from the sample at L (volume voxel coordinates, cell brick b0,
// flagged kCellSkip) along dq (voxels per sample) over cell bricks flagged
// kCellSkip; a super brick (kSuper^3 cell bricks) whose count of cell bricks
// without kCellSkip is 0 is crossed in one step, and so is the block of super
// bricks within distance 1 or 2 of it when their counts are all 0 (the
// neighbour counts of its word).  Returns, in samples from L,
// the end of that run of bricks less m voxels (capped at the domain end less
// m).
__device__ __forceinline__ float skip_run(const VolDev &v, const float L[3], const float dq[3],
                                          const int b0[3], float m)
{
    float tx, ty, tz, dx, dy, dz, tdom = 3.0e38f;
    int sx, sy, sz;
    dda_axis(L[0], dq[0], b0[0], v.r[0], m, tx, dx, sx, tdom);
    dda_axis(L[1], dq[1], b0[1], v.r[1], m, ty, dy, sy, tdom);
    dda_axis(L[2], dq[2], b0[2], v.r[2], m, tz, dz, sz, tdom);
    const float rx = fabsf(dq[0]) * (1.0f / kBrick), ry = fabsf(dq[1]) * (1.0f / kBrick),
                rz = fabsf(dq[2]) * (1.0f / kBrick);
    int bx = b0[0], by = b0[1], bz = b0[2];
    const int nbx = v.nb[0], nby = v.nb[1], nbz = v.nb[2];
    const int max_steps = nbx + nby + nbz + 3;
    float texit = 0.f, dexit = 1.f;
    unsigned sw = super_word(v, bx, by, bz);
    for (int it = 0; it < max_steps; ++it) {
        bool out, new_super;
        if ((sw & kSupCount) == 0u) {
            // to the face of the super brick, or of the empty block around it,
            // every axis advanced to match
            const int reach = (sw & (0xFFu * kSupNear2)) == 0u ? 2 : ((sw & (0xFFu * kSupNear1)) == 0u ? 1 : 0);
            const int nx = inner_faces(bx, sx, reach, nbx), ny = inner_faces(by, sy, reach, nby),
                      nz = inner_faces(bz, sz, reach, nbz);
            const float fx = tx + (float)nx * dx, fy = ty + (float)ny * dy, fz = tz + (float)nz * dz;
            int jx, jy, jz;
            if (fx <= fy && fx <= fz) {
                texit = fx; dexit = fabsf(dq[0]);
                jx = nx + 1; jy = faces_crossed(ty, ry, texit, ny); jz = faces_crossed(tz, rz, texit, nz);
            } else if (fy <= fz) {
                texit = fy; dexit = fabsf(dq[1]);
                jx = faces_crossed(tx, rx, texit, nx); jy = ny + 1; jz = faces_crossed(tz, rz, texit, nz);
            } else {
                texit = fz; dexit = fabsf(dq[2]);
                jx = faces_crossed(tx, rx, texit, nx); jy = faces_crossed(ty, ry, texit, ny); jz = nz + 1;
            }
            bx += sx * jx; tx += (float)jx * dx;
            by += sy * jy; ty += (float)jy * dy;
            bz += sz * jz; tz += (float)jz * dz;
            out = bx < 0 || bx >= nbx || by < 0 || by >= nby || bz < 0 || bz >= nbz;
            new_super = true;
        } else if (tx <= ty && tx <= tz) {
            texit = tx; dexit = fabsf(dq[0]); bx += sx; tx += dx; out = bx < 0 || bx >= nbx;
            new_super = (bx & 3) == (sx > 0 ? 0 : 3);
        } else if (ty <= tz) {
            texit = ty; dexit = fabsf(dq[1]); by += sy; ty += dy; out = by < 0 || by >= nby;
            new_super = (by & 3) == (sy > 0 ? 0 : 3);
        } else {
            texit = tz; dexit = fabsf(dq[2]); bz += sz; tz += dz; out = bz < 0 || bz >= nbz;
            new_super = (bz & 3) == (sz > 0 ? 0 : 3);
        }
        if (out) break;
        const uint8_t cf = __ldg(v.cflag + ((long long)bz * nby + by) * nbx + bx);
        if (new_super) sw = super_word(v, bx, by, bz);
        if ((sw & kSupCount) != 0u && !(cf & kCellSkip)) break;
    }
    return fminf(texit - m * __frcp_rn(dexit), tdom);
}

// Ray state of one volume: camera lattice point and fraction, the direction
// in voxels, and (after the domain is known) the grid step dq = dirv * Delta.
__device__ __forceinline__ void vol_ray(const VolDev &v, const VolFrame &vf, const float d[3], VolRay &vr,
                                        float dirv[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vr.fr[a] = vf.cam_frac[a];
        vr.oi[a] = vf.cam_int[a] - v.h[a];
        dirv[a] = d[a] * v.inv_s;
    }
}

__device__ __forceinline__ float grid_step(const VolDev &v, const FrameParams &P, float dn)
{
    return P.ray_step * v.s / dn;
}

// March one ray through one volume; updates `best` when this volume's hit is
// nearer (or equally near with a lower id).
//
// Step-over rule: a sample can end a bracket only if it is valid with F <= 0,
// which needs an observed voxel with F <= 0 among its cell's corners.  Inside
// a run of cell bricks flagged kCellSkip no such voxel exists, so no sample in
// the run can end a bracket, and the march state after the run is fixed by
// the run's last sample alone.  The march therefore jumps to that last sample
// (at least m voxels inside the run) and evaluates it normally: the result is
// that of the dense march, not an approximation.
//
// Step-over policy: stepping over a run and walking through it sample by
// sample (each sample decided by its cell masks) end in the same state, so
// whether a run is stepped over changes the cost, never the result.  A DDA
// taken by a few lanes of a warp holds the other lanes, and runs met after a
// landing are often short, so with cell masks a later run is stepped over
// only kSkipGap samples after the last landing, or while at most kSkipLanes
// lanes of the warp are still marching (the warp's stragglers).  Without
// masks a walk evaluates every sample, so every run is stepped over.
constexpr int kSkipGap = 48;
constexpr int kSkipLanes = 8;

template <int FMT, typename Off>
__device__ void march_volume(const VolDev &v, const VolFrame &vf, const FrameParams &P,
                             const float d[3], float dn, int slot, Hit &best, RayCount &rc)
{
    const Geo<Off> g = make_geo<Off>(v);
    VolRay vr;
    float dirv[3];
    vol_ray(v, vf, d, vr, dirv);
    // domain [h_t, h_t + r - 1] in camera-relative coordinates
    float lo = P.z_min, hi = P.z_max;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float bmin = (float)(-vr.oi[a]) - vr.fr[a];
        const float bmax = (float)(v.r[a] - 1 - vr.oi[a]) - vr.fr[a];
        if (dirv[a] == 0.f) {
            if (bmin > 0.f || bmax < 0.f) return;
            continue;
        }
        const float inv = 1.0f / dirv[a];
        float t0 = bmin * inv, t1 = bmax * inv;
        if (t0 > t1) { const float tt = t0; t0 = t1; t1 = tt; }
        lo = fmaxf(lo, t0);
        hi = fminf(hi, t1);
    }
    if (!(lo <= hi)) return;
    if (lo > best.tau) return;  // cannot beat the current nearest hit
    const float Delta = grid_step(v, P, dn);
#pragma unroll
    for (int a = 0; a < 3; ++a) vr.dq[a] = dirv[a] * Delta;
    const float k0 = ceilf(lo / Delta), k1 = floorf(hi / Delta);
    if (!(k1 >= k0)) return;
    // integer trip count: bounded even where float k would stop advancing
    // (the domain spans at most sqrt(3) * 8192 / (1/64) grid steps)
    const int nk = (int)fminf(k1 - k0, 1.0e6f);
    const float m = 1e-3f;  // safety margin (voxels) of the step-over rule

    int state = 0;  // 0: no valid previous sample, 1: previous valid > 0, -1: previous valid <= 0
    float Fprev = 0.f;
    bool prev_read = false;  // Fprev holds the previous sample's value (not decided by its mask)
    int cur_b = -1;
    int last_land = -kSkipGap;  // the first run is always stepped over
    for (int kk = 0; kk <= nk; ++kk) {
        const int lanes = __popc(__activemask());
        float k = k0 + (float)kk;
        float rr[3];
        int cell[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) rr[a] = fmaf(k, vr.dq[a], vr.fr[a]);
        locate_cell(v, vr, rr, cell);
        // brick of the sample's cell (its lower corner)
        int bidx = ((cell[2] >> 3) * g.nby + (cell[1] >> 3)) * (int)g.nb0 + (cell[0] >> 3);
        if (bidx != cur_b) {
            cur_b = bidx;
            const bool may_skip = !v.cmask || kk - last_land >= kSkipGap || lanes <= kSkipLanes;
            if (may_skip && (__ldg(v.cflag + bidx) & kCellSkip)) {
                float L[3];
                int bi[3];
                bool inside = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    L[a] = (float)vr.oi[a] + rr[a];
                    bi[a] = cell[a] >> 3;
                    inside &= (L[a] >= (float)(bi[a] * kBrick) + m) &
                              (L[a] <= (float)min(bi[a] * kBrick + kBrick, v.r[a] - 1) - m);
                }
                if (inside) {
                    const float run = skip_run(v, L, vr.dq, bi, m);
                    const int jump = (int)fminf(floorf(run), (float)(nk - kk));
                    if (jump > 0) {
                        // land on the run's last sample and evaluate it below
                        kk += jump;
                        k = k0 + (float)kk;
#pragma unroll
                        for (int a = 0; a < 3; ++a) rr[a] = fmaf(k, vr.dq[a], vr.fr[a]);
                        locate_cell(v, vr, rr, cell);
                        cur_b = ((cell[2] >> 3) * g.nby + (cell[1] >> 3)) * (int)g.nb0 + (cell[0] >> 3);
                        bidx = cur_b;
                        state = 0;
                        last_land = kk;
                        ++rc.skips;
                    }
                }
            }
        }
        if (v.cmask) {
            // a cell without an observed corner with F <= 0 cannot end a
            // bracket (its interpolant is > 0 where valid): the march state
            // follows from its "all corners observed" bit alone
            const ulonglong2 cm = __ldg(v.cmask + (size_t)bidx * 8 + (cell[2] & 7));
            const int bit = ((cell[1] & 7) << 3) | (cell[0] & 7);
            if (!((cm.y >> bit) & 1ull)) {
                state = ((cm.x >> bit) & 1ull) ? 1 : 0;
                prev_read = false;
                continue;
            }
        }
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[a] = rr[a] - (float)(cell[a] - vr.oi[a]);
        const Corners<Off> c = cell_corners(g, cell[0], cell[1], cell[2]);
        bool valid;
        const float F = trilinear<FMT>(v, c, f[0], f[1], f[2], valid);
        ++rc.samples;
        if (!valid) { state = 0; prev_read = false; continue; }
        if (state == 1 && F <= 0.f) {
            // bracket (k-1, k]: bisection on the interpolant, then a secant step
            if (!prev_read) {
                bool pv;
                Fprev = eval_at<FMT>(v, g, vr, k - 1.0f, pv);
            }
            float a = k - 1.0f, b = k, ga = Fprev, gb = F;
            // the corners of the cell last read stay in registers: a midpoint in
            // the same cell re-reads no memory (same arithmetic as trilinear)
            int c0 = -1, c1 = 0, c2 = 0;
            float Fc0 = 0.f, Fc1 = 0.f, Fc2 = 0.f, Fc3 = 0.f, Fc4 = 0.f, Fc5 = 0.f, Fc6 = 0.f, Fc7 = 0.f;
            for (int it = 0; it < P.n_bisect; ++it) {
                const float mid = 0.5f * (a + b);
                if (mid <= a || mid >= b) break;  // interval at float resolution
                float rm[3], fm[3];
                int cm[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) rm[e] = fmaf(mid, vr.dq[e], vr.fr[e]);
                locate(v, vr, rm, cm, fm);
                if (cm[0] != c0 || cm[1] != c1 || cm[2] != c2) {
                    c0 = cm[0];
                    c1 = cm[1];
                    c2 = cm[2];
                    const Corners<Off> q = cell_corners(g, c0, c1, c2);
                    float Wd;
                    load_fw<FMT>(v, q.base, Fc0, Wd);
                    load_fw<FMT>(v, q.base + q.ox, Fc1, Wd);
                    load_fw<FMT>(v, q.base + q.oy, Fc2, Wd);
                    load_fw<FMT>(v, q.base + q.ox + q.oy, Fc3, Wd);
                    load_fw<FMT>(v, q.base + q.oz, Fc4, Wd);
                    load_fw<FMT>(v, q.base + q.ox + q.oz, Fc5, Wd);
                    load_fw<FMT>(v, q.base + q.oy + q.oz, Fc6, Wd);
                    load_fw<FMT>(v, q.base + q.ox + q.oy + q.oz, Fc7, Wd);
                }
                const float x00 = fmaf(fm[0], Fc1 - Fc0, Fc0);
                const float x10 = fmaf(fm[0], Fc3 - Fc2, Fc2);
                const float x01 = fmaf(fm[0], Fc5 - Fc4, Fc4);
                const float x11 = fmaf(fm[0], Fc7 - Fc6, Fc6);
                const float y0 = fmaf(fm[1], x10 - x00, x00);
                const float y1 = fmaf(fm[1], x11 - x01, x01);
                const float gm = fmaf(fm[2], y1 - y0, y0);
                if (gm > 0.f) { a = mid; ga = gm; } else { b = mid; gb = gm; }
            }
            const float den = ga - gb;
            const float ks = den > 0.f ? fmaf(b - a, ga / den, a) : 0.5f * (a + b);
            const float tau = ks * Delta;
            if (tau < best.tau || (tau == best.tau && v.id < best.id)) {
                best.tau = tau;
                best.id = v.id;
                best.slot = slot;
                best.ks = ks;
            }
            return;
        }
        state = (F > 0.f) ? 1 : -1;
        Fprev = F;
        prev_read = true;
    }
}

__device__ __forceinline__ void add_counts(Stats *stats, unsigned rays, unsigned samples,
                                           unsigned skips, unsigned hits)
{
    // one atomic per counter per warp (all lanes call this)
    unsigned long long a = rays, b = samples, c = skips, e = hits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
        e += __shfl_down_sync(0xffffffffu, e, o);
    }
    if ((threadIdx.x & 31) == 0 && stats) {
        if (a) atomicAdd(&stats->rays, a);
        if (b) atomicAdd(&stats->ray_samples, b);
        if (c) atomicAdd(&stats->ray_skips, c);
        if (e) atomicAdd(&stats->ray_hits, e);
    }
}

__device__ __forceinline__ void trace_pixel(const VolDev *__restrict__ vols,
                                            const VolFrame *__restrict__ vfs, const int *list, int n,
                                            const FrameParams &P, const RayOut &out, int merge,
                                            int px, int py, RayCount &rc)
{
    const float dc0 = ((float)px - P.cx) / P.fx, dc1 = ((float)py - P.cy) / P.fy;
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = P.Rf[3 * a] * dc0 + P.Rf[3 * a + 1] * dc1 + P.Rf[3 * a + 2];
    const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);

    Hit best;
    best.tau = FLT_MAX;
    best.id = INT_MAX;
    best.slot = -1;
    best.ks = 0.f;
    const size_t p = (size_t)py * P.width + px;
    if (merge && out.depth[p] > 0.f) {
        best.tau = out.depth[p];
        best.id = out.vol_id[p];
        best.slot = -2;  // existing entry
    }
    // candidate volumes: the table slots list[0, n) (null list: slots 0..n-1);
    // with a view list the order is nearest first, so pruning by the current
    // best hit skips most of the farther ones
    for (int j = 0; j < n; ++j) {
        const int i = list ? list[j] : j;
        const VolDev &v = vols[i];
        // no observed voxel with F <= 0 anywhere in the volume: no sample can
        // end a bracket, so the volume cannot contribute a hit
        if (v.surf && __ldg(v.surf) == 0u) continue;
        const VolFrame vf = vfs[i];
        const bool narrow = v.nbricks * kBrickVox <= 0xFFFFFFFFll;
        if (narrow) {
            switch (v.fmt) {
            case MV_TSDF_F32: march_volume<MV_TSDF_F32, uint32_t>(v, vf, P, d, dn, i, best, rc); break;
            case MV_TSDF_F16: march_volume<MV_TSDF_F16, uint32_t>(v, vf, P, d, dn, i, best, rc); break;
            default: march_volume<MV_TSDF_I16, uint32_t>(v, vf, P, d, dn, i, best, rc); break;
            }
        } else {
            switch (v.fmt) {
            case MV_TSDF_F32: march_volume<MV_TSDF_F32, long long>(v, vf, P, d, dn, i, best, rc); break;
            case MV_TSDF_F16: march_volume<MV_TSDF_F16, long long>(v, vf, P, d, dn, i, best, rc); break;
            default: march_volume<MV_TSDF_I16, long long>(v, vf, P, d, dn, i, best, rc); break;
            }
        }
    }
    if (best.slot == -2) {  // merge: the existing entry (a hit) stays
        ++rc.hits;
        return;
    }
    const bool hit = best.slot >= 0;
    rc.hits += hit ? 1u : 0u;
    // normal and colour of the nearest hit, in its volume's grid
    Shade sh;
    sh.n[0] = sh.n[1] = sh.n[2] = 0.f;
    sh.rgba = 0u;
    if (hit) {
        const VolDev &v = vols[best.slot];
        VolRay vr;
        float dirv[3];
        vol_ray(v, vfs[best.slot], d, vr, dirv);
        const float Delta = grid_step(v, P, dn);
#pragma unroll
        for (int a = 0; a < 3; ++a) vr.dq[a] = dirv[a] * Delta;
        if (v.nbricks * kBrickVox <= 0xFFFFFFFFll) {
            const Geo<uint32_t> g = make_geo<uint32_t>(v);
            switch (v.fmt) {
            case MV_TSDF_F32: shade<MV_TSDF_F32>(v, g, vr, best.ks, sh); break;
            case MV_TSDF_F16: shade<MV_TSDF_F16>(v, g, vr, best.ks, sh); break;
            default: shade<MV_TSDF_I16>(v, g, vr, best.ks, sh); break;
            }
        } else {
            const Geo<long long> g = make_geo<long long>(v);
            switch (v.fmt) {
            case MV_TSDF_F32: shade<MV_TSDF_F32>(v, g, vr, best.ks, sh); break;
            case MV_TSDF_F16: shade<MV_TSDF_F16>(v, g, vr, best.ks, sh); break;
            default: shade<MV_TSDF_I16>(v, g, vr, best.ks, sh); break;
            }
        }
    }
    if (out.depth) out.depth[p] = hit ? best.tau : 0.f;
    if (out.vol_id) out.vol_id[p] = hit ? best.id : -1;
    if (out.normal) {
        out.normal[3 * p + 0] = sh.n[0];
        out.normal[3 * p + 1] = sh.n[1];
        out.normal[3 * p + 2] = sh.n[2];
    }
    if (out.rgba) out.rgba[p] = sh.rgba;
    if (out.vertex) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            out.vertex[3 * p + a] = hit ? P.tf[a] + best.tau * d[a] : 0.f;
    }
}

// Can a ray of the pixel rectangle [x0, x1] x [y0, y1] hit volume v?  False
// only when the volume's domain [h_t, h_t + r - 1] lies wholly outside one
// face of the rectangle's viewing pyramid (widened by half a pixel and a
// rounding margin) or beyond z_max, or when the volume holds no observed
// voxel with F <= 0 (no sample can end a bracket there).  Camera frame,
// this volume's voxel units, camera position split as in the march.
__device__ __forceinline__ bool tile_sees_volume(const VolDev &v, const VolFrame &vf, const FrameParams &P,
                                                 int x0, int x1, int y0, int y1)
{
    if (v.surf && __ldg(v.surf) == 0u) return false;
    const float kl = ((float)x0 - 0.5f - P.cx) / P.fx, kr = ((float)x1 + 0.5f - P.cx) / P.fx;
    const float kt = ((float)y0 - 0.5f - P.cy) / P.fy, kb = ((float)y1 + 0.5f - P.cy) / P.fy;
    const float zfar = P.z_max * v.inv_s + 1.0f;
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = (float)(v.h[a] - vf.cam_int[a]) - vf.cam_frac[a];
        hi[a] = (float)(v.h[a] + v.r[a] - 1 - vf.cam_int[a]) - vf.cam_frac[a];
    }
    bool in_near = false, in_l = false, in_r = false, in_t = false, in_b = false, in_far = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float x = (c & 1) ? hi[0] : lo[0];
        const float y = (c & 2) ? hi[1] : lo[1];
        const float z = (c & 4) ? hi[2] : lo[2];
        const float X = P.Rf[0] * x + P.Rf[3] * y + P.Rf[6] * z;
        const float Y = P.Rf[1] * x + P.Rf[4] * y + P.Rf[7] * z;
        const float Z = P.Rf[2] * x + P.Rf[5] * y + P.Rf[8] * z;
        const float m = 1e-4f * (fabsf(X) + fabsf(Y) + fabsf(Z)) + 1e-3f;
        in_near |= Z > -m;
        in_l |= X - kl * Z > -m;
        in_r |= kr * Z - X > -m;
        in_t |= Y - kt * Z > -m;
        in_b |= kb * Z - Y > -m;
        in_far |= !(Z > zfar + m);
    }
    return in_near && in_l && in_r && in_t && in_b && in_far;
}

// Pixel tiles (128 threads per CTA, selected by the autotuner):
//   0: 16x8 CTA of 2x2 warps, each warp an 8x4 tile
//   1: 32x4 CTA of 4x1 warps, each warp an 8x4 tile
//   2: 8x16 CTA of 1x4 warps, each warp an 8x4 tile
//   3: 32x4 CTA of 1x4 warps, each warp a 32x1 row
template <int TILE>
struct Tile {
    static constexpr int W = (TILE == 0) ? 16 : (TILE == 2) ? 8 : 32;
    static constexpr int H = 128 / W;
    __device__ static void pixel(int w, int lane, int &x, int &y)
    {
        if (TILE == 0) { x = (w & 1) * 8 + (lane & 7); y = (w >> 1) * 4 + (lane >> 3); }
        else if (TILE == 1) { x = w * 8 + (lane & 7); y = lane >> 3; }
        else if (TILE == 2) { x = lane & 7; y = w * 4 + (lane >> 3); }
        else { x = lane; y = w; }
    }
};

template <int TILE>
__device__ __forceinline__ void raycast_tile(const VolDev *__restrict__ vols, const VolFrame *__restrict__ vfs,
                                             int nvol, const FrameParams &P, const RayOut &out, int merge,
                                             Stats *__restrict__ stats, const VisList *__restrict__ vl)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tx, ty;
    Tile<TILE>::pixel(w, lane, tx, ty);
    const int x0 = blockIdx.x * Tile<TILE>::W, y0 = blockIdx.y * Tile<TILE>::H;
    const int px = x0 + tx;
    const int py = y0 + ty;
    const bool active = px < P.width && py < P.height;

    // candidate volumes of this CTA's pixel rectangle, compacted in order (a
    // single volume in view is marched directly: its per-ray tests prune it
    // as the tile test would, without the CTA's barriers)
    __shared__ int s_list[kTileVolMax];
    __shared__ int s_warp[4];
    const int x1 = min(x0 + Tile<TILE>::W, P.width) - 1, y1 = min(y0 + Tile<TILE>::H, P.height) - 1;
    const int n = vl ? vl->count : nvol;
    int total = 0;
    for (int j0 = 0; n > 1 && j0 < n; j0 += 128) {
        const int j = j0 + (int)threadIdx.x;
        int i = 0;
        bool keep = false;
        if (j < n) {
            i = vl ? vl->slot[j] : j;
            keep = tile_sees_volume(vols[i], vfs[i], P, x0, x1, y0, y1);
        }
        const unsigned b = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[w] = __popc(b);
        __syncthreads();
        int off = total;
        for (int k = 0; k < w; ++k) off += s_warp[k];
        if (keep) {
            const int pos = off + __popc(b & ((1u << lane) - 1u));
            if (pos < kTileVolMax) s_list[pos] = i;
        }
        total += s_warp[0] + s_warp[1] + s_warp[2] + s_warp[3];
        __syncthreads();
    }
    // the CTA's candidates when they fit in shared memory, else the view list
    const bool fits = n > 1 && total <= kTileVolMax;
    const int *list = fits ? s_list : (vl ? vl->slot : nullptr);

    RayCount rc{0u, 0u, 0u};
    if (active) trace_pixel(vols, vfs, list, fits ? total : n, P, out, merge, px, py, rc);
    add_counts(stats, active ? 1u : 0u, rc.samples, rc.skips, rc.hits);
}

template <int TILE>
__global__ void __launch_bounds__(128, 6) raycast_kernel(const VolDev *__restrict__ vols,
                                                         const VolFrame *__restrict__ vfs, int nvol,
                                                         FrameParams P, RayOut out, int merge,
                                                         Stats *__restrict__ stats,
                                                         const VisList *__restrict__ vl)
{
    raycast_tile<TILE>(vols, vfs, nvol, P, out, merge, stats, vl);
}

// Several views in one launch (blockIdx.z = view): the view's parameters are
// staged in shared memory, its camera constants are vfs + z * nvol, its view
// list vl + z, and its maps start z * width * height pixels into each output.
template <int TILE>
__global__ void __launch_bounds__(128, 6) raycast_batch_kernel(const VolDev *__restrict__ vols,
                                                               const VolFrame *__restrict__ vfs, int nvol,
                                                               const FrameParams *__restrict__ Pb, RayOut out,
                                                               Stats *__restrict__ stats,
                                                               const VisList *__restrict__ vl)
{
    __shared__ FrameParams s_P;
    static_assert(sizeof(FrameParams) % 4 == 0 && sizeof(FrameParams) / 4 <= 128, "FrameParams staging");
    const int z = blockIdx.z;
    if (threadIdx.x < sizeof(FrameParams) / 4)
        reinterpret_cast<int *>(&s_P)[threadIdx.x] = reinterpret_cast<const int *>(Pb + z)[threadIdx.x];
    __syncthreads();
    const size_t px = (size_t)s_P.width * (size_t)s_P.height * (size_t)z;
    RayOut o = out;
    if (o.depth) o.depth += px;
    if (o.normal) o.normal += 3 * px;
    if (o.rgba) o.rgba += px;
    if (o.vertex) o.vertex += 3 * px;
    if (o.vol_id) o.vol_id += px;
    raycast_tile<TILE>(vols, vfs + (size_t)z * nvol, nvol, s_P, o, 0, stats, vl ? vl + z : nullptr);
}

static const void *raycast_fn(int tile)
{
    switch (tile) {
    case 1: return (const void *)raycast_kernel<1>;
    case 2: return (const void *)raycast_kernel<2>;
    case 3: return (const void *)raycast_kernel<3>;
    default: return (const void *)raycast_kernel<0>;
    }
}

static dim3 raycast_grid(int tile, int width, int height)
{
    const int tw = (tile == 0) ? 16 : (tile == 2) ? 8 : 32;
    const int th = 128 / tw;
    return dim3((width + tw - 1) / tw, (height + th - 1) / th);
}

// Graph node of the raycast of all volumes, after `dep`, reusing the camera
// constants and view list that the frame's setup node computed for the same
// view (the integration changes neither).
cudaError_t graph_raycast(cudaGraph_t g, cudaGraphExec_t exec, cudaGraphNode_t *node, cudaGraphNode_t dep,
                          const VolDev *vols, int nvol, VolFrame *vf, const FrameParams &P, float *depth,
                          float *normal, uint8_t *rgba, float *vertex, int *vol_id, Stats *stats, int tile,
                          VisList *vis)
{
    RayOut o{depth, normal, reinterpret_cast<uint32_t *>(rgba), vertex, vol_id};
    NodeArgs<const VolDev *, const VolFrame *, int, FrameParams, RayOut, int, Stats *, const VisList *> a(
        vols, vf, nvol, P, o, 0, stats, vis);
    return graph_node(g, exec, node, dep, a.params(raycast_fn(tile), raycast_grid(tile, P.width, P.height), 128));
}

cudaError_t launch_raycast(const VolDev *vols, const VolFrame *vfs, int nvol, const FrameParams &P,
                           float *depth, float *normal, uint8_t *rgba, float *vertex, int *vol_id,
                           int merge, Stats *stats, int tile, cudaStream_t s, const VisList *vis)
{
    RayOut o{depth, normal, reinterpret_cast<uint32_t *>(rgba), vertex, vol_id};
    const dim3 grid = raycast_grid(tile, P.width, P.height);
    switch (tile) {
    case 1: raycast_kernel<1><<<grid, 128, 0, s>>>(vols, vfs, nvol, P, o, merge, stats, vis); break;
    case 2: raycast_kernel<2><<<grid, 128, 0, s>>>(vols, vfs, nvol, P, o, merge, stats, vis); break;
    case 3: raycast_kernel<3><<<grid, 128, 0, s>>>(vols, vfs, nvol, P, o, merge, stats, vis); break;
    default: raycast_kernel<0><<<grid, 128, 0, s>>>(vols, vfs, nvol, P, o, merge, stats, vis); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_raycast_batch(const VolDev *vols, const VolFrame *vfs, int nvol, const FrameParams *Pb,
                                 int n_views, int width, int height, float *depth, float *normal, uint8_t *rgba,
                                 float *vertex, int *vol_id, Stats *stats, int tile, cudaStream_t s,
                                 const VisList *vis)
{
    RayOut o{depth, normal, reinterpret_cast<uint32_t *>(rgba), vertex, vol_id};
    dim3 grid = raycast_grid(tile, width, height);
    grid.z = (unsigned)n_views;
    switch (tile) {
    case 1: raycast_batch_kernel<1><<<grid, 128, 0, s>>>(vols, vfs, nvol, Pb, o, stats, vis); break;
    case 2: raycast_batch_kernel<2><<<grid, 128, 0, s>>>(vols, vfs, nvol, Pb, o, stats, vis); break;
    case 3: raycast_batch_kernel<3><<<grid, 128, 0, s>>>(vols, vfs, nvol, Pb, o, stats, vis); break;
    default: raycast_batch_kernel<0><<<grid, 128, 0, s>>>(vols, vfs, nvol, Pb, o, stats, vis); break;
    }
    return cudaGetLastError();
}

}  // namespace mv
