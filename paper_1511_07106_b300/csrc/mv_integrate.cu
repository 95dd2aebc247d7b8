// mv_integrate.cu -- projective TSDF + colour integration (sm_103a).
//
// Sec. Volumetric Integration / Algorithm 1 (first loop) of Salvato, Finman,
// Leonard, arXiv 1511.07106.  The paper sweeps one thread per (x, y) column
// over z for every voxel of every volume.  Here the sweep is restricted to
// the 8x8x8 bricks of all resident volumes that intersect the camera
// frustum: a work list is compacted on the device (brick_list_kernel) and a
// persistent kernel (integrate_kernel) streams each listed brick through
// registers: 4 voxels per thread, 128 threads per brick, 16- or 32-byte
// vector loads/stores of contiguous brick storage.  The per-voxel arithmetic
// is the paper's: position t_s = (h_t + t_l) s, projection to the nearest
// pixel, projective distance, truncation, weighted running average.
#include "mv_internal.cuh"

namespace mv {

// ---------------------------------------------------------------------------
// frustum test of a box of voxel positions [lo, hi] given relative to the
// camera in one volume's voxel units (conservative: never drops a box that
// holds a voxel the per-voxel test would update, nor a sample of a ray)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool box_visible(const float lo[3], const float hi[3], const FrameParams &P,
                                            float inv_s, float z_far)
{
    // plane coefficients (camera frame, voxel units); inside when >= 0
    const float kl = (P.cx + 0.5f) / P.fx, kr = ((float)P.width - 0.5f - P.cx) / P.fx;
    const float kt = (P.cy + 0.5f) / P.fy, kb = ((float)P.height - 0.5f - P.cy) / P.fy;
    // a voxel beyond the farthest accepted depth by more than mu is never updated
    const float zfar = z_far * inv_s + P.trunc_vox;
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
        in_l |= X + kl * Z > -m;
        in_r |= kr * Z - X > -m;
        in_t |= Y + kt * Z > -m;
        in_b |= kb * Z - Y > -m;
        in_far |= !(Z > zfar + m);
    }
    return in_near && in_l && in_r && in_t && in_b && in_far;
}

// Where a brick lies against the depths of the pixels it can project to
// (bounded by the projected corners, all in front of the camera, widened by
// one pixel; their largest and smallest depth come from the smallest pyramid
// level whose tiles are at least as large as that range, or from the
// coarsest level for ranges up to twice its tile):
//   kDepthBehind: every voxel lies farther than every accepted depth by more
//     than mu (sdf = (D - z) |p_c| / z < -mu, as |p_c| / z >= 1), or none
//     projects into the image: the frame updates none of them;
//   kDepthFront: every voxel lies nearer than every accepted depth by more
//     than mu: each voxel it updates gets f = min(1, sdf / mu) = 1, no colour;
//   kDepthFull: kDepthFront, and every voxel projects into the image onto a
//     pixel with an accepted depth (the widened range lies inside the image
//     and no tile of it holds a pixel without one): each voxel is updated
//     with f = 1;
//   kDepthMixedClean: neither of the above, but every voxel projects into the
//     image onto a pixel with an accepted depth (the voxel's own distance
//     test decides);
//   kDepthMixed: otherwise.
// Conservative: margins far above the float rounding of the per-voxel test.
constexpr int kDepthMixed = 0, kDepthBehind = 1, kDepthFront = 2, kDepthFull = 3, kDepthMixedClean = 4;
__device__ __forceinline__ int brick_depth_class(const float lo[3], const float hi[3], const FrameParams &P,
                                                 float inv_s, const unsigned *__restrict__ pyr)
{
    float u0 = 3.0e38f, u1 = -3.0e38f, v0 = 3.0e38f, v1 = -3.0e38f, zmin = 3.0e38f, zmax = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float x = (c & 1) ? hi[0] : lo[0];
        const float y = (c & 2) ? hi[1] : lo[1];
        const float z = (c & 4) ? hi[2] : lo[2];
        const float X = P.Rf[0] * x + P.Rf[3] * y + P.Rf[6] * z;
        const float Y = P.Rf[1] * x + P.Rf[4] * y + P.Rf[7] * z;
        const float Z = P.Rf[2] * x + P.Rf[5] * y + P.Rf[8] * z;
        if (!(Z > 0.5f)) return kDepthMixed;  // at or behind the camera plane
        const float iz = 1.0f / Z;
        const float u = fminf(1.0e6f, fmaxf(-1.0e6f, fmaf(P.fx * X, iz, P.cx)));
        const float v = fminf(1.0e6f, fmaxf(-1.0e6f, fmaf(P.fy * Y, iz, P.cy)));
        u0 = fminf(u0, u); u1 = fmaxf(u1, u);
        v0 = fminf(v0, v); v1 = fmaxf(v1, v);
        zmin = fminf(zmin, Z);
        zmax = fmaxf(zmax, Z);
    }
    const int rx0 = (int)floorf(u0 + 0.5f) - 1, rx1 = (int)floorf(u1 + 0.5f) + 1;
    const int ry0 = (int)floorf(v0 + 0.5f) - 1, ry1 = (int)floorf(v1 + 0.5f) + 1;
    const bool within = rx0 >= 0 && ry0 >= 0 && rx1 < P.width && ry1 < P.height;
    const int x0 = max(0, rx0), x1 = min(P.width - 1, rx1);
    const int y0 = max(0, ry0), y1 = min(P.height - 1, ry1);
    if (x0 > x1 || y0 > y1) return kDepthBehind;  // no voxel projects into the image
    const int span = max(x1 - x0, y1 - y0) + 1;
    int l = 0;
    while (l < kPyrLevels - 1 && (8 << l) < span) ++l;
    // up to two coarsest tiles wide (at most 3 x 3 of them read); wider ranges
    // (bricks close to the camera) keep the frame-wide far test only
    if ((8 << l) * 2 < span) return kDepthMixed;
    const long long off = pyr_level_off(P.width, P.height, l);
    const unsigned *lev_max = pyr + off;
    const unsigned *lev_min = pyr + pyr_level_off(P.width, P.height, kPyrLevels) + off;
    const int nx = pyr_tiles(P.width, l), sh = 3 + l;
    float dmax = 0.f, dmin = 3.0e38f;
    unsigned holes = 0u;  // sign bits: a tile holds a pixel without an accepted depth
    for (int ty = y0 >> sh; ty <= (y1 >> sh); ++ty)
        for (int tx = x0 >> sh; tx <= (x1 >> sh); ++tx) {
            dmax = fmaxf(dmax, __uint_as_float(__ldg(lev_max + (long long)ty * nx + tx)));
            const unsigned wmin = __ldg(lev_min + (long long)ty * nx + tx);
            holes |= wmin;
            dmin = fminf(dmin, __uint_as_float(wmin & 0x7FFFFFFFu));
        }
    if (zmin > fmaf(dmax, inv_s, P.trunc_vox) + 1e-4f * zmin + 1e-3f) return kDepthBehind;
    if (fminf(dmin, 3.0e37f) * inv_s - zmax > P.trunc_vox + 1e-4f * zmax + 1e-3f)
        return within && !(holes >> 31) ? kDepthFull : kDepthFront;
    return within && !(holes >> 31) ? kDepthMixedClean : kDepthMixed;
}

// The box of voxels n * bi .. n * bi + n - 1 per axis (clipped to the volume):
// 0 when the frame updates none of them; 1 when it may; 2 when it may and
// every voxel lies in front of every depth of its pixels by more than mu; 3
// when, besides, every voxel projects onto an accepted depth (all updated);
// 4 when it may, and every voxel projects onto an accepted depth.
__device__ __forceinline__ int box_class(const VolDev &v, const VolFrame &f, const FrameParams &P, int n,
                                         const int bi[3], float z_far, const unsigned *__restrict__ pyr)
{
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int l = bi[a] * n;
        const int u = min(l + n - 1, v.r[a] - 1);
        lo[a] = (float)(v.h[a] + l - f.cam_int[a]) - f.cam_frac[a];
        hi[a] = (float)(v.h[a] + u - f.cam_int[a]) - f.cam_frac[a];
    }
    if (!box_visible(lo, hi, P, v.inv_s, z_far)) return 0;
    if (!pyr) return 1;
    const int cls = brick_depth_class(lo, hi, P, v.inv_s, pyr);
    return cls == kDepthBehind ? 0 : (cls == kDepthFront ? 2 : (cls == kDepthFull ? 3 : (cls == kDepthMixedClean ? 4 : 1)));
}

// 0: not listed; 1: listed; 2: listed, in front of every depth by more than mu;
// 3: listed, every voxel updated with f = 1; 4: listed, every voxel projects
// onto an accepted depth
__device__ __forceinline__ int brick_visible(const VolDev &v, const VolFrame &f,
                                             const FrameParams &P, int bx, int by, int bz, float z_far,
                                             const unsigned *__restrict__ pyr)
{
    const int bi[3] = {bx, by, bz};
    return box_class(v, f, P, kBrick, bi, z_far, pyr);
}

// ---------------------------------------------------------------------------
// per-call setup (one CTA): camera position in every volume's voxel units,
// the work-list counter, and optionally the list of volumes in view
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) frame_setup_kernel(const VolDev *__restrict__ vols, int nvol,
                                                          FrameParams P, VolFrame *__restrict__ vf,
                                                          unsigned *__restrict__ counter,
                                                          VisList *__restrict__ vis)
{
    __shared__ float s_key[kVisSortMax];
    __shared__ unsigned char s_vis[kMaxVolumes];
    for (int v = threadIdx.x; v < nvol; v += blockDim.x) {
        const VolDev &vd = vols[v];
        const double s = (double)vd.s;
        VolFrame f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double q = P.t[a] / s;
            const double fl = floor(q);
            f.cam_int[a] = (int)fl;
            f.cam_frac[a] = (float)(q - fl);
        }
        vf[v] = f;
        if (vis) {
            float lo[3], hi[3], d2 = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = (float)(vd.h[a] - f.cam_int[a]) - f.cam_frac[a];
                hi[a] = (float)(vd.h[a] + vd.r[a] - 1 - f.cam_int[a]) - f.cam_frac[a];
                const float e = fmaxf(fmaxf(lo[a], -hi[a]), 0.f) * vd.s;  // metres outside the box
                d2 += e * e;
            }
            s_vis[v] = box_visible(lo, hi, P, vd.inv_s, P.z_max) ? 1 : 0;
            if (nvol <= kVisSortMax) s_key[v] = d2;
        }
    }
    if (threadIdx.x == 0 && counter) {
        counter[0] = 0u;  // work-list length
        counter[1] = 0u;  // bits of the frame's largest accepted depth (depth_max_kernel)
        counter[2] = 0u;  // bricks whose voxel masks the integration changed
        counter[3] = 0u;  // super bricks in view (the two-level work list)
    }
    if (!vis) return;
    __syncthreads();
    if (nvol <= kVisSortMax) {
        // nearest first: rank of each visible volume by (distance, slot)
        for (int v = threadIdx.x; v < nvol; v += blockDim.x) {
            if (!s_vis[v]) continue;
            int rank = 0;
            for (int u = 0; u < nvol; ++u)
                rank += s_vis[u] && (s_key[u] < s_key[v] || (s_key[u] == s_key[v] && u < v));
            vis->slot[rank] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int n = 0;
            for (int u = 0; u < nvol; ++u) n += s_vis[u];
            long long acc = 0, sacc = 0;
            for (int i = 0; i < n; ++i) {
                const VolDev &vd = vols[vis->slot[i]];
                vis->base[i] = acc;
                vis->sbase[i] = sacc;
                acc += vd.nbricks;
                sacc += (long long)vd.nsb[0] * vd.nsb[1] * vd.nsb[2];
            }
            vis->base[n] = acc;
            vis->sbase[n] = sacc;
            vis->count = n;
            vis->total = acc;
            vis->stotal = sacc;
        }
    } else if (threadIdx.x == 0) {
        int n = 0;
        long long acc = 0, sacc = 0;
        for (int u = 0; u < nvol; ++u) {
            if (!s_vis[u]) continue;
            vis->slot[n] = u;
            vis->base[n] = acc;
            vis->sbase[n] = sacc;
            acc += vols[u].nbricks;
            sacc += (long long)vols[u].nsb[0] * vols[u].nsb[1] * vols[u].nsb[2];
            ++n;
        }
        vis->base[n] = acc;
        vis->sbase[n] = sacc;
        vis->count = n;
        vis->total = acc;
        vis->stotal = sacc;
    }
}

// One thread per brick; warp-aggregated append of visible bricks.
// Bricks are indexed globally over [gb_begin, gb_begin + total) by the
// prefix sums brick_base of the table.
__global__ void __launch_bounds__(256) brick_list_kernel(const VolDev *__restrict__ vols, int nvol,
                                                         const VolFrame *__restrict__ vfs,
                                                         FrameParams P, long long gb_begin,
                                                         long long total_all, uint2 *__restrict__ list,
                                                         unsigned *__restrict__ counter,
                                                         const VisList *__restrict__ vl,
                                                         const unsigned *__restrict__ dmax_bits,
                                                         const unsigned *__restrict__ pyr)
{
    const int lane = threadIdx.x & 31;
    const float z_far = dmax_bits ? fminf(P.z_max, __uint_as_float(*dmax_bits)) : P.z_max;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // with a view list, only the bricks of volumes in view are examined
    const long long total = vl ? vl->total : total_all;
    const int nvis = vl ? vl->count : 0;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
         base += stride) {
        const long long g = base + lane;
        bool vis = false;
        int v = 0;
        unsigned packed = 0;
        if (g < total) {
            long long gb;
            if (vl) {
                int lo = 0, hi = nvis - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (vl->base[mid] <= g) lo = mid; else hi = mid - 1;
                }
                v = vl->slot[lo];
                gb = vols[v].brick_base + (g - vl->base[lo]);
            } else {
                gb = gb_begin + g;
                int lo = 0, hi = nvol - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (vols[mid].brick_base <= gb) lo = mid; else hi = mid - 1;
                }
                v = lo;
            }
            const VolDev &vd = vols[v];
            const unsigned b = (unsigned)(gb - vd.brick_base);  // < 2^30 bricks per volume
            const unsigned bx = b % (unsigned)vd.nb[0];
            const unsigned byz = b / (unsigned)vd.nb[0];
            const unsigned by = byz % (unsigned)vd.nb[1];
            const unsigned bz = byz / (unsigned)vd.nb[1];
            const int cls = brick_visible(vd, vfs[v], P, (int)bx, (int)by, (int)bz, z_far, pyr);
            vis = cls != 0;
            packed = bx | (by << 10) | (bz << 20) | (cls == 2 || cls == 3 ? kListFree : 0u) | (cls >= 3 ? kListFull : 0u);
        }
        const unsigned mask = __ballot_sync(0xffffffffu, vis);
        unsigned pos = 0;
        if (lane == 0 && mask) pos = atomicAdd(counter, (unsigned)__popc(mask));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (vis) list[pos + __popc(mask & ((1u << lane) - 1u))] = make_uint2((unsigned)v, packed);
    }
}

// Two-level work list of the volumes in view (the batched calls).  First one
// thread per super brick (kSuper^3 bricks): the same frustum and depth-tile
// tests on its box, which holds every brick of it, so a super brick that
// fails them holds no brick that passes (both tests only widen with the box:
// more corners on the inside of each plane, a wider pixel range whose depth
// range holds the smaller one's).  The super bricks that pass are listed
// (table slot, sx | sy << 10 | sz << 20).
__global__ void __launch_bounds__(256) super_list_kernel(const VolDev *__restrict__ vols,
                                                         const VolFrame *__restrict__ vfs, FrameParams P,
                                                         uint2 *__restrict__ slist, unsigned *__restrict__ scounter,
                                                         const VisList *__restrict__ vl,
                                                         const unsigned *__restrict__ dmax_bits,
                                                         const unsigned *__restrict__ pyr)
{
    const int lane = threadIdx.x & 31;
    const float z_far = dmax_bits ? fminf(P.z_max, __uint_as_float(*dmax_bits)) : P.z_max;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long total = vl->stotal;
    const int nvis = vl->count;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
         base += stride) {
        const long long g = base + lane;
        bool vis = false;
        int v = 0;
        unsigned packed = 0;
        if (g < total) {
            int lo = 0, hi = nvis - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (vl->sbase[mid] <= g) lo = mid; else hi = mid - 1;
            }
            v = vl->slot[lo];
            const VolDev &vd = vols[v];
            const unsigned si = (unsigned)(g - vl->sbase[lo]);  // < 2^24 super bricks per volume
            const int si3[3] = {(int)(si % (unsigned)vd.nsb[0]), (int)((si / (unsigned)vd.nsb[0]) % (unsigned)vd.nsb[1]),
                                (int)(si / ((unsigned)vd.nsb[0] * (unsigned)vd.nsb[1]))};
            vis = box_class(vd, vfs[v], P, kSuper * kBrick, si3, z_far, pyr) != 0;
            packed = (unsigned)si3[0] | ((unsigned)si3[1] << 10) | ((unsigned)si3[2] << 20);
        }
        const unsigned mask = __ballot_sync(0xffffffffu, vis);
        unsigned pos = 0;
        if (lane == 0 && mask) pos = atomicAdd(scounter, (unsigned)__popc(mask));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (vis) slist[pos + __popc(mask & ((1u << lane) - 1u))] = make_uint2((unsigned)v, packed);
    }
}

// Then one thread per brick of each listed super brick, tested and listed as
// by brick_list_kernel.
__global__ void __launch_bounds__(256) brick_list_super_kernel(const VolDev *__restrict__ vols,
                                                               const VolFrame *__restrict__ vfs, FrameParams P,
                                                               const uint2 *__restrict__ slist,
                                                               const unsigned *__restrict__ scounter,
                                                               uint2 *__restrict__ list, unsigned *__restrict__ counter,
                                                               const unsigned *__restrict__ dmax_bits,
                                                               const unsigned *__restrict__ pyr)
{
    constexpr int kPer = kSuper * kSuper * kSuper;
    const int lane = threadIdx.x & 31;
    const float z_far = dmax_bits ? fminf(P.z_max, __uint_as_float(*dmax_bits)) : P.z_max;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long total = (long long)kPer * (*scounter);
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
         base += stride) {
        const long long g = base + lane;
        bool vis = false;
        unsigned v = 0, packed = 0;
        if (g < total) {
            const uint2 it = slist[g / kPer];
            const int l = (int)(g % kPer);
            v = it.x;
            const VolDev &vd = vols[v];
            const int bx = (int)(it.y & 1023u) * kSuper + (l % kSuper);
            const int by = (int)((it.y >> 10) & 1023u) * kSuper + ((l / kSuper) % kSuper);
            const int bz = (int)(it.y >> 20) * kSuper + l / (kSuper * kSuper);
            if (bx < vd.nb[0] && by < vd.nb[1] && bz < vd.nb[2]) {
                const int cls = brick_visible(vd, vfs[v], P, bx, by, bz, z_far, pyr);
                vis = cls != 0;
                packed = (unsigned)bx | ((unsigned)by << 10) | ((unsigned)bz << 20) | (cls == 2 || cls == 3 ? kListFree : 0u) | (cls >= 3 ? kListFull : 0u);
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, vis);
        unsigned pos = 0;
        if (lane == 0 && mask) pos = atomicAdd(counter, (unsigned)__popc(mask));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (vis) list[pos + __popc(mask & ((1u << lane) - 1u))] = make_uint2(v, packed);
    }
}

// Largest accepted depth of the frame (bits of a non-negative float, so the
// integer maximum is the float maximum); zeroed by the setup kernel.
__global__ void __launch_bounds__(256) depth_max_kernel(const float *__restrict__ depth, int n,
                                                        FrameParams P, unsigned *__restrict__ out)
{
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float D = __ldg(depth + i);
        if (D > 0.f && D >= P.z_min && D <= P.z_max) m = fmaxf(m, D);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// The depth-tile pyramids of the frame (one CTA per 32 x 32 pixels) and its
// largest accepted depth (bits in *out, zeroed by the setup kernel).  The
// accepted depths are positive floats, ordered like their bits.
__global__ void __launch_bounds__(256) depth_tiles_kernel(const float *__restrict__ depth, FrameParams P,
                                                          unsigned *__restrict__ pyr, unsigned *__restrict__ out)
{
    constexpr unsigned kInf = 0x7F800000u, kHole = 0x80000000u;
    // level 0: the block's 4 x 4 tiles of 8 x 8 pixels (largest, smallest
    // depth, and kHole where a pixel inside the image has no accepted depth)
    __shared__ unsigned s_t[4][4], s_n[4][4], s_h[4][4];
    __shared__ unsigned s_1[2][2], s_1n[2][2];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t < 16) {
        s_t[t >> 2][t & 3] = 0u;
        s_n[t >> 2][t & 3] = kInf;
        s_h[t >> 2][t & 3] = 0u;
    }
    __syncthreads();
    // warp w reads rows w + 8 i (tile row i) of the block, lane = column
    const int x = blockIdx.x * 32 + lane;
    float m[4], n[4];
    bool hole[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        m[i] = 0.f;
        n[i] = __uint_as_float(kInf);
        hole[i] = false;
        const int y = blockIdx.y * 32 + w + 8 * i;
        if (x < P.width && y < P.height) {
            const float D = __ldg(depth + (size_t)y * P.width + x);
            if (D > 0.f && D >= P.z_min && D <= P.z_max) m[i] = n[i] = D;
            else hole[i] = true;
        }
    }
    // the 8 columns of a tile are 8 consecutive lanes; the 8 warps meet in shared memory
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float v = m[i], u = n[i];
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            u = fminf(u, __shfl_xor_sync(0xffffffffu, u, o));
        }
        const bool h = (__ballot_sync(0xffffffffu, hole[i]) >> (lane & 24)) & 0xFFu;  // the tile's 8 lanes
        if ((lane & 7) == 0) {
            if (v > 0.f) atomicMax(&s_t[i][lane >> 3], __float_as_uint(v));
            if (__float_as_uint(u) != kInf) atomicMin(&s_n[i][lane >> 3], __float_as_uint(u));
            if (h) atomicOr(&s_h[i][lane >> 3], kHole);
        }
    }
    __syncthreads();
    const long long min_off = pyr_level_off(P.width, P.height, kPyrLevels);  // the smallest-depth pyramid
    if (t < 16) {
        const int tx = blockIdx.x * 4 + (t & 3), ty = blockIdx.y * 4 + (t >> 2);
        if (tx < pyr_tiles(P.width, 0) && ty < pyr_tiles(P.height, 0)) {
            const long long i = (long long)ty * pyr_tiles(P.width, 0) + tx;
            pyr[i] = s_t[t >> 2][t & 3];
            pyr[min_off + i] = s_n[t >> 2][t & 3] | s_h[t >> 2][t & 3];
        }
    } else if (t < 20) {
        const int k = t - 16, lx = k & 1, ly = k >> 1;
        const unsigned mx = max(max(s_t[2 * ly][2 * lx], s_t[2 * ly][2 * lx + 1]),
                                max(s_t[2 * ly + 1][2 * lx], s_t[2 * ly + 1][2 * lx + 1]));
        const unsigned mn = min(min(s_n[2 * ly][2 * lx], s_n[2 * ly][2 * lx + 1]),
                                min(s_n[2 * ly + 1][2 * lx], s_n[2 * ly + 1][2 * lx + 1])) |
                            s_h[2 * ly][2 * lx] | s_h[2 * ly][2 * lx + 1] | s_h[2 * ly + 1][2 * lx] |
                            s_h[2 * ly + 1][2 * lx + 1];
        s_1[ly][lx] = mx;
        s_1n[ly][lx] = mn;
        const int tx = blockIdx.x * 2 + lx, ty = blockIdx.y * 2 + ly;
        if (tx < pyr_tiles(P.width, 1) && ty < pyr_tiles(P.height, 1)) {
            const long long i = pyr_level_off(P.width, P.height, 1) + (long long)ty * pyr_tiles(P.width, 1) + tx;
            pyr[i] = mx;
            pyr[min_off + i] = mn;
        }
    }
    __syncthreads();
    if (t == 0) {
        const unsigned mx = max(max(s_1[0][0], s_1[0][1]), max(s_1[1][0], s_1[1][1]));
        // the hole bit survives the minimum of the low 31 bits
        const unsigned hl = (s_1n[0][0] | s_1n[0][1] | s_1n[1][0] | s_1n[1][1]) & kHole;
        const unsigned mn = min(min(s_1n[0][0] & ~kHole, s_1n[0][1] & ~kHole),
                                min(s_1n[1][0] & ~kHole, s_1n[1][1] & ~kHole)) | hl;
        const long long i = pyr_level_off(P.width, P.height, 2) + (long long)blockIdx.y * pyr_tiles(P.width, 2) + blockIdx.x;
        pyr[i] = mx;
        pyr[min_off + i] = mn;
        if (mx) atomicMax(out, mx);
    }
}

// ---------------------------------------------------------------------------
// integration of one brick by a 128-thread CTA
// ---------------------------------------------------------------------------
struct VoxelUpdate {
    float f[4];      // truncated distance of this frame (units of mu)
    int pix[4];      // pixel index (colour lookup)
    unsigned upd;    // bit j: voxel j updated
    unsigned band;   // bit j: voxel j within the colour band
    unsigned inside; // bit j: voxel j inside the volume (not padding)
};

// CLEAN (kListFull without kListFree): every voxel is known to project into
// the image onto an accepted depth, so those tests are left out.
template <bool CLEAN>
__device__ __forceinline__ void project_voxels(const VolDev &v, const VolFrame &fr,
                                               const FrameParams &P, int bx, int by, int bz,
                                               const float *__restrict__ depth, VoxelUpdate &u, bool front)
{
    const int t = threadIdx.x;
    const int lx0 = (t & 1) * 4, ly = (t >> 1) & 7, lz = t >> 4;
    const int gx = bx * kBrick + lx0, gy = by * kBrick + ly, gz = bz * kBrick + lz;
    // voxel position relative to the camera, in voxel units: exact lattice
    // difference minus the camera's sub-voxel fraction
    const int ix = v.h[0] + gx - fr.cam_int[0];
    const float ry = (float)(v.h[1] + gy - fr.cam_int[1]) - fr.cam_frac[1];
    const float rz = (float)(v.h[2] + gz - fr.cam_int[2]) - fr.cam_frac[2];
    // camera coordinates p_c = R^T (p_w - t), every voxel from its own exact
    // lattice offset by the same expression: a voxel gets the same value in
    // every volume of its pitch, whichever group of 4 holds it (the tiling
    // invariance; a per-group increment X0 + j R would round differently)
    const float KX = fmaf(P.Rf[3], ry, P.Rf[6] * rz);
    const float KY = fmaf(P.Rf[4], ry, P.Rf[7] * rz);
    const float KZ = fmaf(P.Rf[5], ry, P.Rf[8] * rz);
    const float mu = P.trunc_vox, inv_mu = 1.0f / P.trunc_vox;
    const bool row_in = gy < v.r[1] && gz < v.r[2];
    u.upd = u.band = u.inside = 0u;
    // three phases so that the four depth loads are in flight together:
    // projections, loads (pixel 0 stands in for voxels that project nowhere),
    // then the distance and gating
    float Xj[4], Yj[4], Zj[4], izj[4];
    int pj[4];
    bool okj[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float rxj = (float)(ix + j) - fr.cam_frac[0];
        const float X = fmaf(P.Rf[0], rxj, KX);
        const float Y = fmaf(P.Rf[1], rxj, KY);
        const float Z = fmaf(P.Rf[2], rxj, KZ);
        const bool in = row_in && gx + j < v.r[0];
        if (in) u.inside |= 1u << j;
        const float iz = __fdividef(1.0f, Z);  // ~2 ulp; decisions near pixel edges are margins
        const float uf = fmaf(P.fx * X, iz, P.cx);
        const float vf = fmaf(P.fy * Y, iz, P.cy);
        const int ui = __float2int_rd(uf + 0.5f), vi = __float2int_rd(vf + 0.5f);
        const bool ok = CLEAN ? in : in && (Z > 0.f) && (unsigned)ui < (unsigned)P.width && (unsigned)vi < (unsigned)P.height;
        Xj[j] = X;
        Yj[j] = Y;
        Zj[j] = Z;
        izj[j] = iz;
        okj[j] = ok;
        pj[j] = ok ? vi * P.width + ui : 0;
    }
    float Dj[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) Dj[j] = __ldg(depth + pj[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        u.f[j] = 0.f;
        u.pix[j] = 0;
        const float D = Dj[j];
        if (!okj[j] || (!CLEAN && (!(D > 0.f) || D < P.z_min || D > P.z_max))) continue;
        if (front) {
            // the brick lies nearer than every depth of its pixels by more
            // than mu: sdf >= mu, so f = 1 and no colour, as computed below
            u.f[j] = 1.0f;
            u.upd |= 1u << j;
            continue;
        }
        const float X = Xj[j], Y = Yj[j], Z = Zj[j];
        // projective distance along the voxel's ray, in voxels
        const float n2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
        const float lam = n2 * rsqrtf(n2) * izj[j];  // |p_c| / z
        const float sdf = (D * v.inv_s - Z) * lam;
        if (sdf < -mu) continue;
        u.f[j] = fminf(1.0f, sdf * inv_mu);
        u.pix[j] = pj[j];
        u.upd |= 1u << j;
        if (fabsf(sdf) < mu) u.band |= 1u << j;
    }
}

// A brick listed with kListFull and kListFree: every voxel projects onto an
// accepted depth nearer than it by more than mu, so each voxel inside the
// volume takes f = 1 and no colour, as project_voxels would find voxel by
// voxel.
__device__ __forceinline__ void full_front_voxels(const VolDev &v, int bx, int by, int bz, VoxelUpdate &u)
{
    const int t = threadIdx.x;
    const int gx = bx * kBrick + (t & 1) * 4, gy = by * kBrick + ((t >> 1) & 7), gz = bz * kBrick + (t >> 4);
    const bool row_in = gy < v.r[1] && gz < v.r[2];
    unsigned in = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (row_in && gx + j < v.r[0]) in |= 1u << j;
        u.f[j] = 1.0f;
        u.pix[j] = 0;
    }
    u.inside = u.upd = in;
    u.band = 0u;
}

// Division by the invariant divisors d = 2 (w + 1), w = 0..255, as a
// multiplication (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994): with M = ceil(2^32 / d) = (2^32 + e) / d,
// 0 <= e < d, n M / 2^32 = n / d + n e / (d 2^32), and for n < 2^17 the
// added term is below 2^-15 while the fractional part of n / d is at most
// 1 - 1/512, so floor(n M / 2^32) = floor(n / d) exactly.
__device__ __forceinline__ unsigned colour_rcp(int w)
{
    const unsigned long long d = 2ull * (unsigned long long)(w + 1);
    return (unsigned)(((1ull << 32) + d - 1) / d);
}

__device__ __forceinline__ uint32_t blend_rgba(uint32_t old, const uint8_t *__restrict__ rgb, int p,
                                               int cw_max, const unsigned *__restrict__ rcp)
{
    const int wc = (int)(old >> 24);
    const unsigned m = rcp[wc];
    uint32_t out = 0u;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const int c = (int)((old >> (8 * ch)) & 0xFFu);
        const int x = (int)__ldg(rgb + 3 * p + ch);
        const int num = c * wc + x;
        // round half up of num / (wc + 1) = floor((2 num + wc + 1) / (2 (wc + 1)))
        const unsigned nc = __umulhi((unsigned)(2 * num + wc + 1), m);
        out |= nc << (8 * ch);
    }
    out |= (uint32_t)min(wc + 1, cw_max) << 24;
    return out;
}

// Where an integration lists the bricks whose voxel masks it changed (count
// null: the volume set keeps no masks or nothing needs the list).
struct MaskOut {
    uint2 *list;
    unsigned *count;
    unsigned stamp_id;
};

// A CTA collects the bricks whose voxel masks it changed in shared memory and
// appends them to the global list in one piece (no atomic round trip on the
// per-brick critical path).
constexpr int kChgBuf = 128;
struct ChgBuf {
    int flag[2];           // "voxel masks changed" of the current and the next brick
    unsigned n;            // entries in `items`
    unsigned base;         // global position of the final flush
    uint2 items[kChgBuf];
};

// Thread 0 only: append the collected entries to the global list.
__device__ __forceinline__ void flush_changed(ChgBuf &cb, const MaskOut &mo)
{
    const unsigned base = atomicAdd(mo.count, cb.n);
    for (unsigned k = 0; k < cb.n; ++k) mo.list[base + k] = cb.items[k];
    cb.n = 0;
}

template <int FMT>
__device__ __forceinline__ void integrate_brick(const VolDev &v, const VolFrame &fr,
                                                const FrameParams &P, unsigned packed,
                                                const float *__restrict__ depth,
                                                const uint8_t *__restrict__ rgb,
                                                unsigned &n_swept,
                                                unsigned &n_upd,
                                                unsigned &n_band,
                                                const MaskOut &mo, uint2 item, ChgBuf &cb, int parity,
                                                const unsigned *__restrict__ rcp)
{
    const int bx = (int)(packed & 1023u), by = (int)((packed >> 10) & 1023u), bz = packed_bz(packed);
    const long long b = (long long)(((unsigned)bz * (unsigned)v.nb[1] + (unsigned)by) * (unsigned)v.nb[0] +
                                    (unsigned)bx);  // < 2^30 bricks per volume
    const int t = threadIdx.x;
    const long long vox0 = b * kBrickVox + 4 * t;  // first of this thread's 4 voxels
    // the brick's old flag byte, read early: thread 0 updates it after the barriers
    const uint8_t old_flag = t == 0 ? v.bflag[b] : 0;
    // issue this thread's 32 (16) bytes of brick storage before the projection
    // so that the HBM latency overlaps the depth-image gather
    float4 a32, c32;
    uint4 a16;
    if (FMT == MV_TSDF_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(reinterpret_cast<const float2 *>(v.fw) + vox0);
        a32 = p[0];
        c32 = p[1];
    } else {
        a16 = *reinterpret_cast<const uint4 *>(reinterpret_cast<const uint32_t *>(v.fw) + vox0);
    }
    VoxelUpdate u;
    if ((packed & kListFull) && (packed & kListFree))
        full_front_voxels(v, bx, by, bz, u);
    else if (packed & kListFull)
        project_voxels<true>(v, fr, P, bx, by, bz, depth, u, false);
    else
        project_voxels<false>(v, fr, P, bx, by, bz, depth, u, (packed & kListFree) != 0u);
    bool all_pos = true;  // every voxel this thread updated is stored > 0
    bool mchg = false;    // the update changed a voxel's "observed" or "F <= 0" bit
    bool pair_chg = false;  // ... of this thread or of its partner (same 8-voxel row)
    unsigned mine = 0u;   // after a change: "observed" bits of the 4 voxels, "F <= 0" bits << 4
    const bool track = mo.count && v.vmask;  // voxel masks kept and changes listed

    {
        const float wmax = P.w_max;
        if (FMT == MV_TSDF_F32) {
            float F[4] = {a32.x, a32.z, c32.x, c32.z}, W[4] = {a32.y, a32.w, c32.y, c32.w};
            if (u.upd) {
                float4 *p = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(v.fw) + vox0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!((u.upd >> j) & 1u)) continue;
                    // (F W + f) / (W + 1) in increment form
                    const float Fn = F[j] + __fdividef(u.f[j] - F[j], W[j] + 1.0f);
                    mchg |= !(W[j] > 0.f) || ((F[j] <= 0.f) != (Fn <= 0.f));
                    W[j] = fminf(W[j] + 1.0f, wmax);
                    F[j] = Fn;
                    all_pos &= Fn > 0.f;
                }
                p[0] = make_float4(F[0], W[0], F[1], W[1]);
                p[1] = make_float4(F[2], W[2], F[3], W[3]);
            }
            if (track) pair_chg = __shfl_xor_sync(0xffffffffu, (int)mchg, 1) || mchg;
            if (pair_chg) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mine |= ((W[j] > 0.f ? 1u : 0u) | ((W[j] > 0.f) & (F[j] <= 0.f) ? 16u : 0u)) << j;
            }
        } else {
            uint32_t q[4] = {a16.x, a16.y, a16.z, a16.w};
            // both codes store F in the low 16 bits with the sign of an int16
            // (a half's sign bit; +-0 and the int16 code 0 compare <= 0)
            if (u.upd) {
                uint4 *p = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(v.fw) + vox0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!((u.upd >> j) & 1u)) continue;
                    float F, W;
                    if (FMT == MV_TSDF_F16) decode_f16(q[j], F, W); else decode_i16(q[j], F, W);
                    const float Fn = F + __fdividef(u.f[j] - F, W + 1.0f);
                    const float Wn = fminf(W + 1.0f, wmax);
                    const uint32_t q0 = q[j];
                    if (FMT == MV_TSDF_F16) {
                        q[j] = encode_f16(Fn, Wn);
                        all_pos &= stored_f16(Fn) > 0.f;
                    } else {
                        q[j] = encode_i16(Fn, Wn);
                        all_pos &= stored_i16(Fn) > 0.f;
                    }
                    mchg |= (q0 >> 16) == 0u || (((short)(q0 & 0xFFFFu) <= 0) != ((short)(q[j] & 0xFFFFu) <= 0));
                }
                *p = make_uint4(q[0], q[1], q[2], q[3]);
            }
            if (track) pair_chg = __shfl_xor_sync(0xffffffffu, (int)mchg, 1) || mchg;
            if (pair_chg) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool obs = (q[j] >> 16) != 0u;
                    mine |= ((obs ? 1u : 0u) | (obs & ((short)(q[j] & 0xFFFFu) <= 0) ? 16u : 0u)) << j;
                }
            }
        }
    }
    // a brick whose voxel masks changed raises its flag in cb.flag[parity]
    // (read after the barriers below; see integrate_kernel for its reset),
    // and each changed 8-voxel row (held by the thread pair 2k, 2k + 1) is
    // stored by the even thread: its "observed" and "F <= 0" bytes
    if (pair_chg) {
        const unsigned other = __shfl_xor_sync(__activemask(), mine, 1);
        if ((t & 1) == 0) {
            uint8_t *row = reinterpret_cast<uint8_t *>(v.vmask + b * 16) + (t >> 1);
            row[0] = (uint8_t)((mine & 0xFu) | ((other & 0xFu) << 4));
            row[64] = (uint8_t)((mine >> 4) | (other & 0xF0u));
        }
        if (mchg) cb.flag[parity] = 1;
    }

    if (u.upd) {
        if (rgb && u.band) {
            uint4 *pc = reinterpret_cast<uint4 *>(v.rgba + vox0);
            uint4 c = *pc;
            uint32_t cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((u.band >> j) & 1u) cc[j] = blend_rgba(cc[j], rgb, u.pix[j], P.color_w_max, rcp);
            *pc = make_uint4(cc[0], cc[1], cc[2], cc[3]);
        }
    }
    const int nu = __popc(u.upd);
    n_swept += __popc(u.inside);
    n_upd += nu;
    if (rgb) n_band += __popc(u.band);

    // brick flag maintenance (exact summaries, see mv_internal.cuh): FREE when
    // every voxel was updated to a positive value, or the brick was FREE and
    // every updated voxel stayed positive; EMPTY while no voxel was ever
    // updated; NONEG like FREE but without requiring every voxel observed
    const int brick_all = __syncthreads_and(u.upd == 0xFu ? 1 : 0);
    if (t == 0) cb.flag[parity ^ 1] = 0;  // the next brick's flag, read by everyone before this barrier
    const int brick_any = __syncthreads_or(u.upd != 0u ? 1 : 0);
    const int brick_pos = __syncthreads_and(all_pos ? 1 : 0);
    if (track && cb.flag[parity]) {
        // the brick is stamped and listed for the cell-mask refresh
        if (t == 0) {
            v.stamp[b] = mo.stamp_id;
            if (cb.n == kChgBuf) flush_changed(cb, mo);
            cb.items[cb.n++] = item;
        }
    }
    if (t == 0) {
        const uint8_t old = old_flag;
        uint8_t nf = 0;
        if (brick_pos && (brick_all || (old & kFlagFree))) nf |= kFlagFree;
        if ((old & kFlagEmpty) && !brick_any) nf |= kFlagEmpty;
        if (brick_pos && (brick_all || (old & kFlagNoNeg))) nf |= kFlagNoNeg;
        if (nf != old) v.bflag[b] = nf;
        if (v.surf && ((old ^ nf) & kFlagNoNeg)) atomicAdd(v.surf, (nf & kFlagNoNeg) ? 0xFFFFFFFFu : 1u);
    }
}

__global__ void __launch_bounds__(128) integrate_kernel(const VolDev *__restrict__ vols,
                                                        const VolFrame *__restrict__ vfs,
                                                        const uint2 *__restrict__ list,
                                                        const unsigned *__restrict__ counter,
                                                        FrameParams P, const float *__restrict__ depth,
                                                        const uint8_t *__restrict__ rgb,
                                                        Stats *__restrict__ stats, MaskOut mo)
{
    __shared__ VolDev s_v;
    __shared__ VolFrame s_f;
    // per-brick "voxel masks changed" flags, used alternately by consecutive
    // bricks: brick k raises cb.flag[k & 1] before its first barrier, reads it
    // after its third, and thread 0 clears cb.flag[(k + 1) & 1] after brick
    // k's first barrier (all reads of it by brick k - 1 are done, no write of
    // brick k + 1 has started)
    __shared__ ChgBuf cb;
    __shared__ unsigned s_rcp[256];  // colour_rcp(w), published by the first volume-change barrier
    for (int w = threadIdx.x; w < 256; w += blockDim.x) s_rcp[w] = colour_rcp(w);
    if (threadIdx.x == 0) {  // published by the first volume-change barrier (or the final one)
        cb.flag[0] = cb.flag[1] = 0;
        cb.n = 0;
    }
    int parity = 0;
    int cached = -1;
    const unsigned n = *counter;
    unsigned n_swept = 0, n_upd = 0, n_band = 0, n_bricks = 0;  // per thread: < 2^32
    for (unsigned i = blockIdx.x; i < n; i += gridDim.x) {
        const uint2 it = list[i];
        // the volume descriptor and camera constants are staged in shared
        // memory once per change of volume (uniform across the CTA)
        if ((int)it.x != cached) {
            __syncthreads();
            if (threadIdx.x < sizeof(VolDev) / 4)
                reinterpret_cast<int *>(&s_v)[threadIdx.x] = reinterpret_cast<const int *>(vols + it.x)[threadIdx.x];
            if (threadIdx.x < sizeof(VolFrame) / 4)
                reinterpret_cast<int *>(&s_f)[threadIdx.x] = reinterpret_cast<const int *>(vfs + it.x)[threadIdx.x];
            __syncthreads();
            cached = (int)it.x;
        }
        const VolDev &v = s_v;
        const VolFrame fr = s_f;
        switch (v.fmt) {
        case MV_TSDF_F32: integrate_brick<MV_TSDF_F32>(v, fr, P, it.y, depth, rgb, n_swept, n_upd, n_band, mo, it, cb, parity, s_rcp); break;
        case MV_TSDF_F16: integrate_brick<MV_TSDF_F16>(v, fr, P, it.y, depth, rgb, n_swept, n_upd, n_band, mo, it, cb, parity, s_rcp); break;
        default: integrate_brick<MV_TSDF_I16>(v, fr, P, it.y, depth, rgb, n_swept, n_upd, n_band, mo, it, cb, parity, s_rcp); break;
        }
        parity ^= 1;
        ++n_bricks;
    }
    if (mo.count) {
        // the CTA's remaining changed bricks, appended together
        __syncthreads();
        if (threadIdx.x == 0 && cb.n) cb.base = atomicAdd(mo.count, cb.n);
        __syncthreads();
        for (unsigned k = threadIdx.x; k < cb.n; k += blockDim.x) mo.list[cb.base + k] = cb.items[k];
    }
    // one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_swept += __shfl_down_sync(0xffffffffu, n_swept, o);
        n_upd += __shfl_down_sync(0xffffffffu, n_upd, o);
        n_band += __shfl_down_sync(0xffffffffu, n_band, o);
    }
    if ((threadIdx.x & 31) == 0 && stats) {
        if (n_swept) atomicAdd(&stats->swept, (unsigned long long)n_swept);
        if (n_upd) atomicAdd(&stats->updated, (unsigned long long)n_upd);
        if (n_band) atomicAdd(&stats->band, (unsigned long long)n_band);
        if (threadIdx.x == 0 && n_bricks) atomicAdd(&stats->bricks, (unsigned long long)n_bricks);
    }
}

// Exact brick flags from the stored voxels (after a host write).
template <int FMT>
__device__ __forceinline__ void voxel_state(const VolDev &v, long long off, bool &valid, bool &pos)
{
    float F, W;
    if (FMT == MV_TSDF_F32) {
        const float2 q = reinterpret_cast<const float2 *>(v.fw)[off];
        F = q.x; W = q.y;
    } else {
        const uint32_t q = reinterpret_cast<const uint32_t *>(v.fw)[off];
        if (FMT == MV_TSDF_F16) decode_f16(q, F, W); else decode_i16(q, F, W);
    }
    valid = W > 0.f;
    pos = F > 0.f;
}

__global__ void __launch_bounds__(128) brick_flags_kernel(VolDev v)
{
    for (long long b = blockIdx.x; b < v.nbricks; b += gridDim.x) {
        bool all_free = true, all_empty = true, no_neg = true;
        for (int k = threadIdx.x; k < kBrickVox; k += blockDim.x) {
            bool valid, pos;
            const long long off = b * kBrickVox + k;
            if (v.fmt == MV_TSDF_F32) voxel_state<MV_TSDF_F32>(v, off, valid, pos);
            else if (v.fmt == MV_TSDF_F16) voxel_state<MV_TSDF_F16>(v, off, valid, pos);
            else voxel_state<MV_TSDF_I16>(v, off, valid, pos);
            all_free &= valid && pos;
            all_empty &= !valid;
            no_neg &= !valid || pos;
        }
        const int f = __syncthreads_and(all_free ? 1 : 0);
        const int e = __syncthreads_and(all_empty ? 1 : 0);
        const int nn = __syncthreads_and(no_neg ? 1 : 0);
        if (threadIdx.x == 0) {
            v.bflag[b] = (uint8_t)((f ? kFlagFree : 0) | (e ? kFlagEmpty : 0) | (nn ? kFlagNoNeg : 0));
            if (!nn && v.surf) atomicAdd(v.surf, 1u);  // zeroed before this kernel
        }
    }
}

// Cell-brick flag of cell brick (cx, cy, cz): the trilinear cells whose lower
// corner lies in that brick read voxels of the 8 bricks (cx, cy, cz) + {0,1}^3;
// bricks beyond the volume only hold cells outside the interpolation domain.
__device__ __forceinline__ bool cell_skip_of(const VolDev &v, int cx, int cy, int cz)
{
    bool skip = true;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int x = cx + (e & 1), y = cy + ((e >> 1) & 1), z = cz + ((e >> 2) & 1);
        if (x < v.nb[0] && y < v.nb[1] && z < v.nb[2])
            skip &= (v.bflag[((long long)z * v.nb[1] + y) * v.nb[0] + x] & kFlagNoNeg) != 0;
    }
    return skip;
}

__device__ __forceinline__ unsigned *super_count_of(const VolDev &v, int cx, int cy, int cz)
{
    return v.sup + ((long long)(cz / kSuper) * v.nsb[1] + cy / kSuper) * v.nsb[0] + cx / kSuper;
}

// The count of super brick (sx, sy, sz) became non-zero (up = true) or zero:
// every super brick within Chebyshev distance kSupReach moves its
// neighbour counts.  Additions and subtractions commute, so the words are
// exact once every change of the kernel has been applied, whatever the
// order (a field may wrap in between; nothing reads them in between).  The
// (2 kSupReach + 1)^3 neighbours k = first, first + stride, ... are done
// here (several threads may share them).
__device__ void super_occupancy_changed(const VolDev &v, int sx, int sy, int sz, bool up, int first, int stride)
{
    constexpr int kSide = 2 * kSupReach + 1;
    for (int k = first; k < kSide * kSide * kSide; k += stride) {
        const int dx = k % kSide - kSupReach, dy = (k / kSide) % kSide - kSupReach, dz = k / (kSide * kSide) - kSupReach;
        const int x = sx + dx, y = sy + dy, z = sz + dz;
        if (x < 0 || y < 0 || z < 0 || x >= v.nsb[0] || y >= v.nsb[1] || z >= v.nsb[2]) continue;
        const int d = max(abs(dx), max(abs(dy), abs(dz)));
        const unsigned inc = (d <= 1 ? kSupNear1 : 0u) + kSupNear2;
        atomicAdd(v.sup + ((long long)z * v.nsb[1] + y) * v.nsb[0] + x, up ? inc : 0u - inc);
    }
}

// Moves the count of the super brick holding cell brick (cx, cy, cz) by one
// (up: a cell brick lost kCellSkip).  The count never drops below zero (a
// decrement follows the increment of the same cell brick), so the returned
// old value tells exactly one thread of each change to or from zero: +1 when
// the count left zero, -1 when it reached zero, else 0.
__device__ __forceinline__ int move_super_count(const VolDev &v, int cx, int cy, int cz, bool up)
{
    const unsigned old = atomicAdd(super_count_of(v, cx, cy, cz), up ? 1u : 0xFFFFFFFFu);
    return (old & kSupCount) == (up ? 0u : 1u) ? (up ? 1 : -1) : 0;
}

// Incremental refresh: the flag byte is changed by an atomic on its aligned
// word, whose returned old value tells exactly one of several threads that
// refresh the same cell brick that the flag changed; that thread moves the
// super-brick count.  Returns move_super_count's change to or from zero
// (the caller updates the neighbour counts).
__device__ __forceinline__ int update_cell_flag(const VolDev &v, int cx, int cy, int cz, bool skip)
{
    uint8_t *pb = v.cflag + ((long long)cz * v.nb[1] + cy) * v.nb[0] + cx;
    if (!v.sup) {
        *pb = skip ? kCellSkip : 0;
        return 0;
    }
    unsigned *w = reinterpret_cast<unsigned *>(reinterpret_cast<uintptr_t>(pb) & ~(uintptr_t)3);
    const unsigned bit = (unsigned)kCellSkip << (8u * (unsigned)(reinterpret_cast<uintptr_t>(pb) & 3u));
    const unsigned old = skip ? atomicOr(w, bit) : atomicAnd(w, ~bit);
    return ((old & bit) != 0u) != skip ? move_super_count(v, cx, cy, cz, !skip) : 0;
}

// Row z (0..7) of the voxel mask `plane` (0 observed, 1 observed with F <= 0)
// of brick (bx, by, bz); bricks beyond the volume hold no observed voxel.
__device__ __forceinline__ unsigned long long vmask_row(const VolDev &v, int bx, int by, int bz, int plane,
                                                        int z)
{
    if (bx >= v.nb[0] || by >= v.nb[1] || bz >= v.nb[2]) return 0ull;
    const long long b = ((long long)bz * v.nb[1] + by) * v.nb[0] + bx;
    return __ldg(v.vmask + b * 16 + plane * 8 + z);
}

// Cell masks of slice z of cell brick (cx, cy, cz) from the voxel masks of
// the bricks (cx, cy, cz) + {0,1}^3: the corners of cell (x, y, z) are the
// voxels (x + i, y + j, z + k); the +x / +y / +xy corners of a voxel row are
// the row shifted by one bit / one byte, with the bits that leave the brick
// taken from the neighbour brick's first column / row.
__device__ __forceinline__ ulonglong2 cell_mask_slice(const VolDev &v, int cx, int cy, int cz, int z)
{
    constexpr unsigned long long kCol0 = 0x0101010101010101ull, kCol7 = 0x8080808080808080ull;
    unsigned long long V = ~0ull, N = 0ull;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const int zz = z + dz, bz = cz + (zz >> 3), sz = zz & 7;
#pragma unroll
        for (int plane = 0; plane < 2; ++plane) {
            const unsigned long long a = vmask_row(v, cx, cy, bz, plane, sz);
            const unsigned long long ax = vmask_row(v, cx + 1, cy, bz, plane, sz);
            const unsigned long long ay = vmask_row(v, cx, cy + 1, bz, plane, sz);
            const unsigned long long axy = vmask_row(v, cx + 1, cy + 1, bz, plane, sz);
            const unsigned long long sx = ((a >> 1) & ~kCol7) | ((ax & kCol0) << 7);   // (x + 1, y)
            const unsigned long long ux = ((ay >> 1) & ~kCol7) | ((axy & kCol0) << 7); // (x + 1, y) of +y
            const unsigned long long sy = (a >> 8) | (ay << 56);                      // (x, y + 1)
            const unsigned long long sxy = (sx >> 8) | (ux << 56);                    // (x + 1, y + 1)
            if (plane == 0) V &= a & sx & sy & sxy;
            else N |= a | sx | sy | sxy;
        }
    }
    return make_ulonglong2(V, N);
}

// After an integration, for volumes without cell masks: refresh the
// cell-brick flags that the listed bricks feed (each listed brick b is read
// by the cell bricks b - {0,1}^3) from the brick summaries.
__global__ void __launch_bounds__(256) cell_flags_kernel(const VolDev *__restrict__ vols,
                                                         const uint2 *__restrict__ list,
                                                         const unsigned *__restrict__ counter)
{
    const unsigned long long n = 8ull * (*counter);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        const uint2 it = list[i >> 3];
        const int d = (int)(i & 7);
        const VolDev &v = vols[it.x];
        if (!v.cflag || v.cmask) continue;
        const int cx = (int)(it.y & 1023u) - (d & 1);
        const int cy = (int)((it.y >> 10) & 1023u) - ((d >> 1) & 1);
        const int cz = packed_bz(it.y) - ((d >> 2) & 1);
        if (cx < 0 || cy < 0 || cz < 0) continue;
        const int ch = update_cell_flag(v, cx, cy, cz, cell_skip_of(v, cx, cy, cz));
        if (ch) super_occupancy_changed(v, cx / kSuper, cy / kSuper, cz / kSuper, ch > 0, 0, 1);
    }
}

// After an integration, for volumes with cell masks: the integration listed
// the bricks whose voxel masks changed (and stamped them with stamp_id);
// every cell brick c that reads one of them (c = b - d, d in {0,1}^3) gets its
// cell masks and its flag recomputed, once: by the smallest d for which
// c + d changed.  Each CTA first gives one thread to each of kCellMaskPairs
// (changed brick, d) pairs and collects the cell bricks they own in shared
// memory, then refreshes those with 8 threads each (one per slice), so that
// pairs owned elsewhere hold no lanes during the refresh.
constexpr int kCellMaskCta = 256;
constexpr int kCellMaskPairs = 64;
__global__ void __launch_bounds__(kCellMaskCta) cell_masks_kernel(const VolDev *__restrict__ vols,
                                                                const uint2 *__restrict__ changed,
                                                                const unsigned *__restrict__ counter,
                                                                unsigned stamp_id)
{
    __shared__ uint2 s_item[kCellMaskPairs];  // (table slot, packed cell brick) owned by this CTA
    __shared__ unsigned s_n;
    const unsigned long long n = 8ull * (*counter);
    const int t = threadIdx.x, z = t & 7;
    const unsigned group = 0xFFu << (t & 24);  // the 8 slice threads of one cell brick
    for (unsigned long long base = (unsigned long long)blockIdx.x * kCellMaskPairs; base < n;
         base += (unsigned long long)gridDim.x * kCellMaskPairs) {
        if (t == 0) s_n = 0;
        __syncthreads();
        const unsigned long long i = base + t;
        if (t < kCellMaskPairs && i < n) {
            const uint2 it = changed[i >> 3];
            const int d = (int)(i & 7);
            const VolDev &v = vols[it.x];
            const int cx = (int)(it.y & 1023u) - (d & 1);
            const int cy = (int)((it.y >> 10) & 1023u) - ((d >> 1) & 1);
            const int cz = packed_bz(it.y) - ((d >> 2) & 1);
            bool own = cx >= 0 && cy >= 0 && cz >= 0;
            // not the owner when c + e changed for some e < d (the stamps of
            // all those bricks are loaded together, then tested)
            if (own) {
                unsigned st[7];
#pragma unroll
                for (int e = 0; e < 7; ++e) {
                    const int x = cx + (e & 1), y = cy + ((e >> 1) & 1), w = cz + (e >> 2);
                    const bool in = e < d && x < v.nb[0] && y < v.nb[1] && w < v.nb[2];
                    st[e] = in ? __ldg(v.stamp + ((long long)w * v.nb[1] + y) * v.nb[0] + x) : ~stamp_id;
                }
#pragma unroll
                for (int e = 0; e < 7; ++e) own &= st[e] != stamp_id;
            }
            if (own) s_item[atomicAdd(&s_n, 1u)] = make_uint2(it.x, (unsigned)cx | ((unsigned)cy << 10) | ((unsigned)cz << 20));
        }
        __syncthreads();
        const unsigned m = s_n;
        for (unsigned k = (unsigned)t >> 3; k < m; k += kCellMaskCta / 8) {
            const uint2 it = s_item[k];
            const VolDev &v = vols[it.x];
            const int cx = (int)(it.y & 1023u), cy = (int)((it.y >> 10) & 1023u), cz = (int)(it.y >> 20);
            const long long c = ((long long)cz * v.nb[1] + cy) * v.nb[0] + cx;
            const ulonglong2 mk = cell_mask_slice(v, cx, cy, cz, z);
            v.cmask[c * 8 + z] = mk;
            // the cell brick can be stepped over when none of its cells has an
            // observed corner with F <= 0 (OR of the 8 slices' N rows)
            unsigned long long nz = mk.y;
            nz |= __shfl_xor_sync(group, nz, 1);
            nz |= __shfl_xor_sync(group, nz, 2);
            nz |= __shfl_xor_sync(group, nz, 4);
            int ch = z == 0 ? update_cell_flag(v, cx, cy, cz, nz == 0ull) : 0;
            // a change of the super count to or from zero: the 8 slice threads
            // share the neighbour updates
            ch = __shfl_sync(group, ch, t & 24);
            if (ch) super_occupancy_changed(v, cx / kSuper, cy / kSuper, cz / kSuper, ch > 0, z, 8);
        }
        __syncthreads();
    }
}

// Voxel masks of every brick of one volume from its stored voxels (after a
// host write or a swap-in); 128 threads per brick, one ballot per 4 rows.
__global__ void __launch_bounds__(128) vmask_all_kernel(VolDev v)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long b = blockIdx.x; b < v.nbricks; b += gridDim.x) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = i * 128 + (int)threadIdx.x;  // voxel (k & 7, (k >> 3) & 7, k >> 6)
            bool valid, pos;
            const long long off = b * kBrickVox + k;
            if (v.fmt == MV_TSDF_F32) voxel_state<MV_TSDF_F32>(v, off, valid, pos);
            else if (v.fmt == MV_TSDF_F16) voxel_state<MV_TSDF_F16>(v, off, valid, pos);
            else voxel_state<MV_TSDF_I16>(v, off, valid, pos);
            const unsigned o = __ballot_sync(0xffffffffu, valid);
            const unsigned ng = __ballot_sync(0xffffffffu, valid && !pos);
            if (lane == 0) {
                // 32 voxels = rows 4 (w & 1) .. + 3 of slice 2 i + (w >> 1)
                unsigned *rows = reinterpret_cast<unsigned *>(v.vmask + b * 16);
                const int word = 2 * (2 * i + (w >> 1)) + (w & 1);
                rows[word] = o;
                rows[16 + word] = ng;
            }
        }
    }
}

// Cell masks of every brick of one volume (after vmask_all_kernel).
__global__ void __launch_bounds__(256) cmask_all_kernel(VolDev v)
{
    const long long n = v.nbricks * 8;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const long long b = i >> 3;
        const int z = (int)(i & 7);
        const int cx = (int)(b % v.nb[0]);
        const int cy = (int)((b / v.nb[0]) % v.nb[1]);
        const int cz = (int)(b / ((long long)v.nb[0] * v.nb[1]));
        v.cmask[i] = cell_mask_slice(v, cx, cy, cz, z);
    }
}

// Every cell-brick flag of one volume (after a host write), with the
// super-brick words recounted from zero (zeroed before this kernel).
__global__ void __launch_bounds__(256) cell_flags_all_kernel(VolDev v)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < v.nbricks; b += stride) {
        const int cx = (int)(b % v.nb[0]);
        const int cy = (int)((b / v.nb[0]) % v.nb[1]);
        const int cz = (int)(b / ((long long)v.nb[0] * v.nb[1]));
        const bool skip = cell_skip_of(v, cx, cy, cz);
        v.cflag[b] = skip ? kCellSkip : 0;
        if (!skip && v.sup && move_super_count(v, cx, cy, cz, true))
            super_occupancy_changed(v, cx / kSuper, cy / kSuper, cz / kSuper, true, 0, 1);
    }
}

// ---------------------------------------------------------------------------
// full-cover streaming: brick gather / scatter between the host copy of a
// swapped-out volume (pinned, mapped) and a device staging slot
// ---------------------------------------------------------------------------
// A frame reads, of a staged volume, the bricks holding the cells along the
// pixel rays inside [z_min, z_max] (and the integration's bricks, a subset):
// a cell whose lower corner lies in brick b covers positions [8b, 8b + 8)
// and reads bricks b and b + 1, so brick b' is needed when the box
// [8b' - 8, 8b' + 8] meets the view frustum.  Those bricks are copied from
// the host copy into the slot, one warp per brick; the slot's other bricks
// are never read by the frame's kernels.
__global__ void __launch_bounds__(128) stream_gather_kernel(VolDev v, const VolFrame *__restrict__ vf,
                                                            FrameParams P, const uint4 *__restrict__ h_fw,
                                                            const uint4 *__restrict__ h_rgba,
                                                            unsigned long long *__restrict__ count)
{
    const VolFrame f = *vf;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int fw_vec = kBrickVox * (v.fmt == MV_TSDF_F32 ? 8 : 4) / 16;
    const int col_vec = kBrickVox * 4 / 16;
    uint4 *dfw = reinterpret_cast<uint4 *>(v.fw);
    uint4 *dcol = reinterpret_cast<uint4 *>(v.rgba);
    unsigned long long n = 0;
    for (long long b = warp; b < v.nbricks; b += nwarps) {
        const int bi[3] = {(int)(b % v.nb[0]), (int)((b / v.nb[0]) % v.nb[1]),
                           (int)(b / ((long long)v.nb[0] * v.nb[1]))};
        float lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int l = max(0, bi[a] * kBrick - kBrick), u = min(v.r[a] - 1, bi[a] * kBrick + kBrick);
            lo[a] = (float)(v.h[a] + l - f.cam_int[a]) - f.cam_frac[a];
            hi[a] = (float)(v.h[a] + u - f.cam_int[a]) - f.cam_frac[a];
        }
        if (!box_visible(lo, hi, P, v.inv_s, P.z_max)) continue;
        // all of a lane's loads first (many host reads in flight), then the stores
        uint4 a[8], c[4];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k * 32 < fw_vec) a[k] = h_fw[b * fw_vec + k * 32 + lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = h_rgba[b * col_vec + k * 32 + lane];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k * 32 < fw_vec) dfw[b * fw_vec + k * 32 + lane] = a[k];
#pragma unroll
        for (int k = 0; k < 4; ++k) dcol[b * col_vec + k * 32 + lane] = c[k];
        ++n;
    }
    if (lane == 0 && n) atomicAdd(count, n);
}

// The bricks the integration changed (its work list) back to the host copy.
__global__ void __launch_bounds__(128) stream_scatter_kernel(VolDev v, const uint2 *__restrict__ list,
                                                             const unsigned *__restrict__ counter,
                                                             uint4 *__restrict__ h_fw, uint4 *__restrict__ h_rgba,
                                                             unsigned long long *__restrict__ count)
{
    const unsigned n = *counter;
    const int lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const int fw_vec = kBrickVox * (v.fmt == MV_TSDF_F32 ? 8 : 4) / 16;
    const int col_vec = kBrickVox * 4 / 16;
    const uint4 *sfw = reinterpret_cast<const uint4 *>(v.fw);
    const uint4 *scol = reinterpret_cast<const uint4 *>(v.rgba);
    for (unsigned i = warp; i < n; i += nwarps) {
        const unsigned pk = list[i].y;
        const long long b = ((long long)packed_bz(pk) * v.nb[1] + ((pk >> 10) & 1023u)) * v.nb[0] + (pk & 1023u);
        uint4 a[8], c[4];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k * 32 < fw_vec) a[k] = sfw[b * fw_vec + k * 32 + lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = scol[b * col_vec + k * 32 + lane];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k * 32 < fw_vec) h_fw[b * fw_vec + k * 32 + lane] = a[k];
#pragma unroll
        for (int k = 0; k < 4; ++k) h_rgba[b * col_vec + k * 32 + lane] = c[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(count, (unsigned long long)n);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_frame_setup(const VolDev *vols, int nvol, const FrameParams &P, VolFrame *vf,
                               unsigned *counter, cudaStream_t s, VisList *vis)
{
    frame_setup_kernel<<<1, 256, 0, s>>>(vols, nvol, P, vf, counter, vis);
    return cudaGetLastError();
}

static long long list_blocks(long long total, int num_sms)
{
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return blocks;
}

// With a view list (the batched calls) and a super-brick list buffer
// (slist, total_sup entries, its length in counter[3]): the two-level list;
// otherwise one thread per brick.  The second kernel and its launch cost
// about 3 us; the first saves about 5.5 us per million bricks in view, so the
// callers pass slist from about a million resident bricks on.
cudaError_t launch_brick_list(const VolDev *vols, int nvol, const VolFrame *vfs,
                              const FrameParams &P, long long gb_begin, long long total,
                              uint2 *list, unsigned *counter, int num_sms, cudaStream_t s,
                              const VisList *vis, const unsigned *dmax_bits, const unsigned *pyr,
                              uint2 *slist, long long total_sup)
{
    if (total <= 0) return cudaSuccess;
    if (vis && slist) {
        super_list_kernel<<<(unsigned)list_blocks(total_sup, num_sms), 256, 0, s>>>(
            vols, vfs, P, slist, counter + 3, vis, dmax_bits, pyr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        brick_list_super_kernel<<<(unsigned)num_sms * 8, 256, 0, s>>>(vols, vfs, P, slist, counter + 3, list,
                                                                     counter, dmax_bits, pyr);
        return cudaGetLastError();
    }
    brick_list_kernel<<<(unsigned)list_blocks(total, num_sms), 256, 0, s>>>(
        vols, nvol, vfs, P, gb_begin, total, list, counter, vis, dmax_bits, pyr);
    return cudaGetLastError();
}

static unsigned depth_max_blocks(int n, int num_sms)
{
    int b = (n + 1023) / 1024;
    if (b > num_sms * 2) b = num_sms * 2;
    return (unsigned)(b < 1 ? 1 : b);
}

static dim3 depth_tiles_grid(const FrameParams &P) { return dim3((P.width + 31) / 32, (P.height + 31) / 32); }

// The frame's largest accepted depth, and with pyr its depth-tile pyramid.
cudaError_t launch_depth_max(const float *depth, const FrameParams &P, unsigned *out, int num_sms,
                             cudaStream_t s, unsigned *pyr)
{
    if (pyr) {
        depth_tiles_kernel<<<depth_tiles_grid(P), 256, 0, s>>>(depth, P, pyr, out);
        return cudaGetLastError();
    }
    const int n = P.width * P.height;
    depth_max_kernel<<<depth_max_blocks(n, num_sms), 256, 0, s>>>(depth, n, P, out);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const VolDev *vols, const VolFrame *vfs, const uint2 *list,
                             const unsigned *counter, const FrameParams &P, const float *depth,
                             const uint8_t *rgb, Stats *stats, int grid, cudaStream_t s,
                             uint2 *changed, unsigned *chg_count, unsigned stamp_id)
{
    integrate_kernel<<<grid, 128, 0, s>>>(vols, vfs, list, counter, P, depth, rgb, stats,
                                          MaskOut{changed, chg_count, stamp_id});
    return cudaGetLastError();
}

// Voxel and cell masks of a whole volume from its stored voxels.
cudaError_t launch_mask_rebuild(const VolDev &v, int num_sms, cudaStream_t s)
{
    if (!v.vmask || !v.cmask) return cudaSuccess;
    long long blocks = v.nbricks;
    const long long cap = (long long)num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    vmask_all_kernel<<<(unsigned)blocks, 128, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long cblocks = (v.nbricks * 8 + 255) / 256;
    if (cblocks > cap) cblocks = cap;
    if (cblocks < 1) cblocks = 1;
    cmask_all_kernel<<<(unsigned)cblocks, 256, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_brick_flags(const VolDev &v, int num_sms, cudaStream_t s)
{
    long long blocks = v.nbricks;
    const long long cap = (long long)num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (v.surf) {
        const cudaError_t z = cudaMemsetAsync(v.surf, 0, sizeof(unsigned), s);
        if (z != cudaSuccess) return z;
    }
    if (v.sup) {
        const size_t nsuper = (size_t)v.nsb[0] * v.nsb[1] * v.nsb[2];
        const cudaError_t z = cudaMemsetAsync(v.sup, 0, sizeof(unsigned) * nsuper, s);
        if (z != cudaSuccess) return z;
    }
    brick_flags_kernel<<<(unsigned)blocks, 128, 0, s>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long cblocks = (v.nbricks + 255) / 256;
    if (cblocks > cap) cblocks = cap;
    if (cblocks < 1) cblocks = 1;
    cell_flags_all_kernel<<<(unsigned)cblocks, 256, 0, s>>>(v);
    e = cudaGetLastError();
    if (e != cudaSuccess || !v.vmask) return e;
    return launch_mask_rebuild(v, num_sms, s);
}

cudaError_t launch_cell_flags(const VolDev *vols, const uint2 *list, const unsigned *counter,
                              int num_sms, cudaStream_t s)
{
    cell_flags_kernel<<<num_sms * 4, 256, 0, s>>>(vols, list, counter);
    return cudaGetLastError();
}

cudaError_t launch_cell_masks(const VolDev *vols, const uint2 *changed, const unsigned *counter,
                              unsigned stamp_id, int num_sms, cudaStream_t s)
{
    cell_masks_kernel<<<num_sms * 8, kCellMaskCta, 0, s>>>(vols, changed, counter, stamp_id);
    return cudaGetLastError();
}

cudaError_t frame_setup_node(cudaGraph_t g, cudaGraphExec_t exec, cudaGraphNode_t *node,
                             cudaGraphNode_t dep, const VolDev *vols, int nvol, const FrameParams &P,
                             VolFrame *vf, VisList *vis)
{
    NodeArgs<const VolDev *, int, FrameParams, VolFrame *, unsigned *, VisList *> a(vols, nvol, P, vf, nullptr,
                                                                                  vis);
    return graph_node(g, exec, node, dep, a.params((const void *)frame_setup_kernel, 1, 256));
}

// Graph nodes of one integration: setup -> depth max -> brick list -> integrate -> cell flags.
// Nodes: 0 setup, 1 depth tiles, 2 (and 3) the work list, 4 integration,
// 5 cell-mask refresh.  With slist the work list is two-level (2: super
// bricks, 3: their bricks), else one kernel over total bricks (node 3 unused).
cudaError_t graph_integrate(cudaGraph_t g, cudaGraphExec_t exec, cudaGraphNode_t nodes[6],
                            cudaGraphNode_t dep, const VolDev *vols, int nvol, VolFrame *vf,
                            const FrameParams &P, long long total, long long total_sup, uint2 *slist,
                            uint2 *list, unsigned *counter, const float *depth, const uint8_t *rgb, Stats *stats,
                            int grid_int, int num_sms, VisList *vis, uint2 *changed, unsigned stamp_id,
                            unsigned *pyr)
{
    NodeArgs<const VolDev *, int, FrameParams, VolFrame *, unsigned *, VisList *> a0(vols, nvol, P, vf, counter,
                                                                                   vis);
    cudaError_t e = graph_node(g, exec, &nodes[0], dep, a0.params((const void *)frame_setup_kernel, 1, 256));
    if (e != cudaSuccess) return e;
    NodeArgs<const float *, FrameParams, unsigned *, unsigned *> am(depth, P, pyr, counter + 1);
    e = graph_node(g, exec, &nodes[1], nodes[0], am.params((const void *)depth_tiles_kernel, depth_tiles_grid(P), 256));
    if (e != cudaSuccess) return e;
    if (slist) {
        NodeArgs<const VolDev *, const VolFrame *, FrameParams, uint2 *, unsigned *, const VisList *,
                 const unsigned *, const unsigned *>
            as(vols, vf, P, slist, counter + 3, vis, counter + 1, pyr);
        e = graph_node(g, exec, &nodes[2], nodes[1],
                       as.params((const void *)super_list_kernel, (unsigned)list_blocks(total_sup, num_sms), 256));
        if (e != cudaSuccess) return e;
        NodeArgs<const VolDev *, const VolFrame *, FrameParams, const uint2 *, const unsigned *, uint2 *, unsigned *,
                 const unsigned *, const unsigned *>
            a1(vols, vf, P, slist, counter + 3, list, counter, counter + 1, pyr);
        e = graph_node(g, exec, &nodes[3], nodes[2],
                       a1.params((const void *)brick_list_super_kernel, (unsigned)num_sms * 8, 256));
    } else {
        NodeArgs<const VolDev *, int, const VolFrame *, FrameParams, long long, long long, uint2 *, unsigned *,
                 const VisList *, const unsigned *, const unsigned *>
            a1(vols, nvol, vf, P, 0LL, total, list, counter, vis, counter + 1, pyr);
        e = graph_node(g, exec, &nodes[2], nodes[1],
                       a1.params((const void *)brick_list_kernel, (unsigned)list_blocks(total, num_sms), 256));
    }
    if (e != cudaSuccess) return e;
    NodeArgs<const VolDev *, const VolFrame *, const uint2 *, const unsigned *, FrameParams, const float *,
             const uint8_t *, Stats *, MaskOut>
        a2(vols, vf, list, counter, P, depth, rgb, stats, MaskOut{changed, counter + 2, stamp_id});
    e = graph_node(g, exec, &nodes[4], slist ? nodes[3] : nodes[2],
                   a2.params((const void *)integrate_kernel, grid_int, 128));
    if (e != cudaSuccess) return e;
    NodeArgs<const VolDev *, const uint2 *, const unsigned *, unsigned> a3(vols, changed, counter + 2, stamp_id);
    return graph_node(g, exec, &nodes[5], nodes[4], a3.params((const void *)cell_masks_kernel, num_sms * 8, kCellMaskCta));
}

int integrate_max_ctas_per_sm()
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrate_kernel, 128, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 8;
    return per_sm;
}

int integrate_occupancy_grid(int num_sms) { return num_sms * integrate_max_ctas_per_sm(); }

}  // namespace mv

namespace mv {

// Gather and scatter are bound by the host link, not the SMs: two CTAs per SM
// keep enough reads in flight and leave the SMs to the kernels of the other
// slots, which run at the same time on other streams.
cudaError_t launch_stream_gather(const VolDev &v, const VolFrame *vf, const FrameParams &P, const void *h_fw,
                                 const void *h_rgba, unsigned long long *count, int num_sms, cudaStream_t s)
{
    stream_gather_kernel<<<num_sms * 2, 128, 0, s>>>(v, vf, P, reinterpret_cast<const uint4 *>(h_fw),
                                                     reinterpret_cast<const uint4 *>(h_rgba), count);
    return cudaGetLastError();
}

cudaError_t launch_stream_scatter(const VolDev &v, const uint2 *list, const unsigned *counter, void *h_fw,
                                  void *h_rgba, unsigned long long *count, int num_sms, cudaStream_t s)
{
    stream_scatter_kernel<<<num_sms * 2, 128, 0, s>>>(v, list, counter, reinterpret_cast<uint4 *>(h_fw),
                                                      reinterpret_cast<uint4 *>(h_rgba), count);
    return cudaGetLastError();
}

}  // namespace mv
