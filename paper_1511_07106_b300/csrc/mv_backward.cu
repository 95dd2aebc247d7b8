// mv_backward.cu -- gradients of the raycast (sm_103a).
//
// Not in the paper: the differentiable form of the raycast of Sec. Raycasting,
// used to refine camera poses against rendered depth and colour.  The pose is
// perturbed on the left, T(xi) = exp(xi^) T with xi = (rho, phi) in the world
// frame.  At the hit x* = t + tau* d with the analytic trilinear gradient g of
// the hit cell and its corner weights w_j:
//   dtau/dxi = -(g, x* x g) / (g.d),     dtau/dF_j = -w_j / (g.d),
//   dx*/dxi  = [I | -[x*]_x] + d dtau/dxi,
//   C(x) = sum_j w_j(x) c_j / 255,  dC/dxi = J_C dx*/dxi,  dC/dF_j = J_C d dtau/dF_j.
// The backward pass does not store march samples: it re-derives the hit cell
// from the forward's depth and volume id (one thread per pixel and pose).
// Pixels without a hit, with an unobserved corner, at grazing incidence
// (|g.d| <= 1e-3 |g||d|) or within 1e-3 voxel of a cell face are skipped.
// The pose gradient is summed per CTA and then per pose in a fixed order, so
// it is the same on every run; the TSDF gradients are float atomics.
#include "mv_internal.cuh"

namespace mv {


__device__ __forceinline__ int slot_of(const VolDev *vols, int nvol, int id)
{
    int lo = 0, hi = nvol - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (vols[mid].id < id) lo = mid + 1; else hi = mid;
    }
    return (nvol > 0 && vols[lo].id == id) ? lo : -1;
}

template <int FMT>
__device__ __forceinline__ void corner_fw(const VolDev &v, long long off, float &F, float &W)
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

// Per-pixel gradient terms; returns false for skipped pixels.
template <int FMT>
__device__ bool pixel_grad(const VolDev &v, const float *Tf, const float *cam, float tau, const float d[3],
                           float gdep, const float gc[3], float jpose[6], long long corner_off[8],
                           long long lin[8], float &coef, float w[8])
{
    // hit point in this volume's voxel coordinates, from the camera position
    // (formed in double on the host: B300's FP64 rate is a small fraction of
    // its FP32 rate, so the kernel does no FP64 arithmetic)
    float q[3], xs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q[a] = __ldg(cam + a) + tau * d[a] * v.inv_s;
        xs[a] = __ldg(Tf + 9 + a) + tau * d[a];
    }
    int cell[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(q[a]);
        const int c = max(0, min(v.r[a] - 2, (int)fl));
        cell[a] = c;
        fr[a] = q[a] - (float)c;
        if (fr[a] < 1e-3f || fr[a] > 1.0f - 1e-3f) return false;
    }
    const long long base = vox_offset(v, cell[0], cell[1], cell[2]);
    const long long ox = ((cell[0] & 7) == 7) ? (long long)(kBrickVox - 7) : 1;
    const long long oy = ((cell[1] & 7) == 7) ? (long long)v.nb[0] * kBrickVox - 56 : 8;
    const long long oz = ((cell[2] & 7) == 7) ? (long long)v.nb[0] * v.nb[1] * kBrickVox - 448 : 64;
    float g[3] = {0.f, 0.f, 0.f};
    float JC[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const long long off = base + (dx ? ox : 0) + (dy ? oy : 0) + (dz ? oz : 0);
        corner_off[k] = off;
        lin[k] = ((long long)(cell[2] + dz) * v.r[1] + (cell[1] + dy)) * v.r[0] + (cell[0] + dx);
        float F, W;
        corner_fw<FMT>(v, off, F, W);
        if (!(W > 0.f)) return false;
        const uint32_t col = __ldg(v.rgba + off);
        const float wx = dx ? fr[0] : 1.f - fr[0];
        const float wy = dy ? fr[1] : 1.f - fr[1];
        const float wz = dz ? fr[2] : 1.f - fr[2];
        w[k] = wx * wy * wz;
        const float gw0 = (dx ? 1.f : -1.f) * wy * wz * v.inv_s;
        const float gw1 = wx * (dy ? 1.f : -1.f) * wz * v.inv_s;
        const float gw2 = wx * wy * (dz ? 1.f : -1.f) * v.inv_s;
        g[0] += F * gw0;
        g[1] += F * gw1;
        g[2] += F * gw2;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float c = (float)((col >> (8 * ch)) & 0xFFu) * (1.0f / 255.0f);
            JC[ch][0] += c * gw0;
            JC[ch][1] += c * gw1;
            JC[ch][2] += c * gw2;
        }
    }
    const float gd = g[0] * d[0] + g[1] * d[1] + g[2] * d[2];
    const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(fabsf(gd) > 1e-3f * gn * dn)) return false;
    const float inv_gd = 1.0f / gd;
    float jt[6];
    jt[0] = -g[0] * inv_gd;
    jt[1] = -g[1] * inv_gd;
    jt[2] = -g[2] * inv_gd;
    jt[3] = -(xs[1] * g[2] - xs[2] * g[1]) * inv_gd;
    jt[4] = -(xs[2] * g[0] - xs[0] * g[2]) * inv_gd;
    jt[5] = -(xs[0] * g[1] - xs[1] * g[0]) * inv_gd;
    // u = J_C^T gc (colour upstream pulled back to the hit point)
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = JC[0][a] * gc[0] + JC[1][a] * gc[1] + JC[2][a] * gc[2];
    // dC/dxi^T gc = u^T ([I | -[x*]_x] + d jt^T) = (u, x* x u) + (u.d) jt
    const float ud = u[0] * d[0] + u[1] * d[1] + u[2] * d[2];
    jpose[0] = gdep * jt[0] + u[0] + ud * jt[0];
    jpose[1] = gdep * jt[1] + u[1] + ud * jt[1];
    jpose[2] = gdep * jt[2] + u[2] + ud * jt[2];
    jpose[3] = gdep * jt[3] + (xs[1] * u[2] - xs[2] * u[1]) + ud * jt[3];
    jpose[4] = gdep * jt[4] + (xs[2] * u[0] - xs[0] * u[2]) + ud * jt[4];
    jpose[5] = gdep * jt[5] + (xs[0] * u[1] - xs[1] * u[0]) + ud * jt[5];
    // dL/dF_j = (gdep + u.d) dtau/dF_j = -(gdep + u.d) w_j / gd
    coef = -(gdep + ud) * inv_gd;
    return true;
}

// sign(x) as torch.sign gives it for finite x: -1, 0 or 1
__device__ __forceinline__ float sign_of(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// The L1 loss of pose refinement: the mean over the n_valid pixels valid in
// both renders (depth > 0 in each) of |depth - ref_depth| + colour_weight *
// sum over RGB of |colour - ref_colour|, colour = 8-bit value / 255.  Its
// gradient at a pixel: w = 1 / n_valid where valid (else 0),
// dL/ddepth = sign(ddepth) w, dL/dcolour = (colour_weight sign(dcolour)) w,
// the same operations in the same order as the closed form of the Python
// binding (l1_loss_grad), and the colour signs taken from the 8-bit values,
// so the two give the same bits.  The pixel's inputs (reference depth, both
// colours, n_valid) are loaded with its depth and volume id.
struct L1Pixel {
    float rd;
    uchar4 a, b;
    unsigned n_valid;
};

__device__ __forceinline__ void l1_pixel_grad(const BackwardArgs &A, const L1Pixel &q, float tau, float &gdep,
                                              float gc[3])
{
    const float w = (tau > 0.f && q.rd > 0.f) ? __fdiv_rn(1.f, (float)max(q.n_valid, 1u)) : 0.f;
    gdep = sign_of(tau - q.rd) * w;
    const uchar4 a = q.a, b = q.b;
    const float cw = A.colour_weight;
    gc[0] = (cw * sign_of((float)a.x - (float)b.x)) * w;
    gc[1] = (cw * sign_of((float)a.y - (float)b.y)) * w;
    gc[2] = (cw * sign_of((float)a.z - (float)b.z)) * w;
}

// One pixel's share of the L1 statistics (colours packed R, G, B, A from the
// low byte up).
__device__ __forceinline__ void l1_accumulate(float d, float r, unsigned a, unsigned b, unsigned &cnt, float &ld,
                                              unsigned long long &lc)
{
    if (!(d > 0.f && r > 0.f)) return;
    ++cnt;
    ld += fabsf(d - r);
    lc += (unsigned)(abs((int)(a & 0xFFu) - (int)(b & 0xFFu)) + abs((int)((a >> 8) & 0xFFu) - (int)((b >> 8) & 0xFFu)) +
                     abs((int)((a >> 16) & 0xFFu) - (int)((b >> 16) & 0xFFu)));
}

// Sum over a CTA of 256 threads in a fixed order (warp trees, then the 8
// warps in order); the result is valid in thread 0.
__device__ __forceinline__ void l1_cta_sum(unsigned &cnt, float &ld, unsigned long long &lc)
{
    __shared__ unsigned s_c[8];
    __shared__ unsigned long long s_l[8];
    __shared__ float s_d[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        ld += __shfl_down_sync(0xffffffffu, ld, o);
        lc += __shfl_down_sync(0xffffffffu, lc, o);
    }
    __syncthreads();  // the slots may still be read by a previous sum
    if (lane == 0) {
        s_c[w] = cnt;
        s_d[w] = ld;
        s_l[w] = lc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cnt = 0;
        ld = 0.f;
        lc = 0;
        for (int k = 0; k < 8; ++k) {
            cnt += s_c[k];
            ld += s_d[k];
            lc += s_l[k];
        }
    }
}

// Statistics of the L1 loss over all n pixels of all views: the count of
// pixels valid in both renders and the loss (see l1_pixel_grad; the colour
// term as the exact integer sum of the 8-bit differences, divided by 255
// once).  Four pixels per step with 16-byte loads where the arrays allow
// them.  Per CTA a count, the colour sum and a float sum of the depth
// differences, then the last CTA to finish adds them (its threads a fixed
// stride of CTAs each, then the CTA sum: a fixed order), writes the count to
// state[1] and the loss to *loss, and resets state[0] for the next call.
__global__ void __launch_bounds__(256) l1_stats_kernel(const float *__restrict__ depth,
                                                       const float *__restrict__ ref_depth,
                                                       const uint8_t *__restrict__ rgba,
                                                       const uint8_t *__restrict__ ref_rgba, long long n,
                                                       float colour_weight, unsigned *state, float *loss)
{
    unsigned long long *col_part = reinterpret_cast<unsigned long long *>(state + 2);
    unsigned *cnt_part = state + 2 + 2 * kL1Ctas;
    float *dep_part = reinterpret_cast<float *>(state + 2 + 3 * kL1Ctas);
    unsigned cnt = 0;
    unsigned long long lc = 0;
    float ld = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(depth) | reinterpret_cast<uintptr_t>(ref_depth) |
                       reinterpret_cast<uintptr_t>(rgba) | reinterpret_cast<uintptr_t>(ref_rgba)) & 15u) == 0;
    long long tail = 0;
    if (vec) {
        const long long n4 = n >> 2;
        for (long long q = first; q < n4; q += stride) {
            const float4 d = reinterpret_cast<const float4 *>(depth)[q];
            const float4 r = reinterpret_cast<const float4 *>(ref_depth)[q];
            const uint4 a = reinterpret_cast<const uint4 *>(rgba)[q];
            const uint4 b = reinterpret_cast<const uint4 *>(ref_rgba)[q];
            l1_accumulate(d.x, r.x, a.x, b.x, cnt, ld, lc);
            l1_accumulate(d.y, r.y, a.y, b.y, cnt, ld, lc);
            l1_accumulate(d.z, r.z, a.z, b.z, cnt, ld, lc);
            l1_accumulate(d.w, r.w, a.w, b.w, cnt, ld, lc);
        }
        tail = n4 << 2;
    }
    const unsigned *rgba4 = reinterpret_cast<const unsigned *>(rgba);
    const unsigned *ref4 = reinterpret_cast<const unsigned *>(ref_rgba);
    for (long long i = tail + first; i < n; i += stride) l1_accumulate(depth[i], ref_depth[i], rgba4[i], ref4[i], cnt, ld, lc);
    l1_cta_sum(cnt, ld, lc);
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        cnt_part[blockIdx.x] = cnt;
        col_part[blockIdx.x] = lc;
        dep_part[blockIdx.x] = ld;
        __threadfence();
        s_last = atomicAdd(state, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    cnt = 0;
    lc = 0;
    ld = 0.f;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
        cnt += __ldcg(cnt_part + k);
        lc += __ldcg(col_part + k);
        ld += __ldcg(dep_part + k);
    }
    l1_cta_sum(cnt, ld, lc);
    if (threadIdx.x == 0) {
        const float wgt = __fdiv_rn(1.f, (float)max(cnt, 1u));
        state[1] = cnt;
        *loss = ld * wgt + colour_weight * (((float)lc / 255.f) * wgt);
        state[0] = 0u;
    }
}

cudaError_t launch_l1_stats(const float *depth, const float *ref_depth, const uint8_t *rgba, const uint8_t *ref_rgba,
                            long long n, float colour_weight, unsigned *scratch, float *loss, cudaStream_t s)
{
    l1_stats_kernel<<<kL1Ctas, 256, 0, s>>>(depth, ref_depth, rgba, ref_rgba, n, colour_weight, scratch, loss);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(128) raycast_backward_kernel(BackwardArgs A)
{
    const int p = blockIdx.z;
    const int px = blockIdx.x * 16 + (threadIdx.x & 15);
    const int py = blockIdx.y * 8 + (threadIdx.x >> 4);
    const float *Tf = A.pose_f + 12 * p;
    float jp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (px < A.width && py < A.height) {
        const size_t pix = ((size_t)p * A.height + py) * A.width + px;
        const float tau = A.depth[pix];
        const int id = A.vol_id[pix];
        L1Pixel q1{0.f, make_uchar4(0, 0, 0, 0), make_uchar4(0, 0, 0, 0), 1u};
        if (A.ref_depth) {
            q1.rd = A.ref_depth[pix];
            q1.a = reinterpret_cast<const uchar4 *>(A.rgba)[pix];
            q1.b = reinterpret_cast<const uchar4 *>(A.ref_rgba)[pix];
            q1.n_valid = __ldg(A.l1_count);
        }
        const int slot = (tau > 0.f && id >= 0) ? slot_of(A.vols, A.nvol, id) : -1;
        if (slot >= 0) {
            const VolDev &v = A.vols[slot];
            const float *cam = A.cam_f + 3 * ((size_t)p * A.nvol + slot);
            const float dc0 = ((float)px - A.cx) / A.fx, dc1 = ((float)py - A.cy) / A.fy;
            float d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                d[a] = __ldg(Tf + 3 * a) * dc0 + __ldg(Tf + 3 * a + 1) * dc1 + __ldg(Tf + 3 * a + 2);
            float gdep = A.grad_depth ? A.grad_depth[pix] : 0.f;
            float gc[3] = {0.f, 0.f, 0.f};
            if (A.ref_depth) {
                l1_pixel_grad(A, q1, tau, gdep, gc);
            } else if (A.grad_rgb) {
                gc[0] = A.grad_rgb[3 * pix];
                gc[1] = A.grad_rgb[3 * pix + 1];
                gc[2] = A.grad_rgb[3 * pix + 2];
            }
            long long off[8], lin[8];
            float w[8], coef = 0.f;
            bool ok;
            switch (v.fmt) {
            case MV_TSDF_F32: ok = pixel_grad<MV_TSDF_F32>(v, Tf, cam, tau, d, gdep, gc, jp, off, lin, coef, w); break;
            case MV_TSDF_F16: ok = pixel_grad<MV_TSDF_F16>(v, Tf, cam, tau, d, gdep, gc, jp, off, lin, coef, w); break;
            default: ok = pixel_grad<MV_TSDF_I16>(v, Tf, cam, tau, d, gdep, gc, jp, off, lin, coef, w); break;
            }
            if (!ok) {
#pragma unroll
                for (int k = 0; k < 6; ++k) jp[k] = 0.f;
            } else if (A.grad_tsdf && A.grad_tsdf[slot]) {
                float *gt = A.grad_tsdf[slot];
#pragma unroll
                for (int k = 0; k < 8; ++k) atomicAdd(gt + lin[k], coef * w[k]);
            }
        }
    }
    // pose gradient: warp sums, then the CTA's sum of each component written
    // to its own slot (reduced per pose in a fixed order by pose_sum_kernel;
    // one atomic per warp on the same six addresses serialised in L2)
    __shared__ float s_part[4][6];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float s = jp[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) s_part[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        const size_t per_pose = (size_t)gridDim.x * gridDim.y;
        A.partial[((size_t)p * per_pose + cta) * 6 + k] = ((s_part[0][k] + s_part[1][k]) + s_part[2][k]) + s_part[3][k];
    }
}

// grad_pose[6 p + k] = sum over the CTAs of pose p of their partial sums, in a
// fixed order (one CTA of 256 threads per pose; the same bits on every run)
__global__ void __launch_bounds__(256) pose_sum_kernel(const float *__restrict__ partial, int per_pose,
                                                       float *__restrict__ grad_pose)
{
    __shared__ float s_acc[6][256];
    const int p = blockIdx.x;
    const float *src = partial + (size_t)p * per_pose * 6;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int c = threadIdx.x; c < per_pose; c += blockDim.x)
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] += src[(size_t)c * 6 + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) s_acc[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 6; ++k) s_acc[k][threadIdx.x] += s_acc[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 6) grad_pose[6 * p + threadIdx.x] = s_acc[threadIdx.x][0];
}

// CTAs per pose of the backward kernel (sizes the partial-sum buffer).
size_t backward_ctas_per_pose(int width, int height)
{
    return (size_t)((width + 15) / 16) * (size_t)((height + 7) / 8);
}

cudaError_t launch_raycast_backward(const BackwardArgs &A, cudaStream_t s)
{
    dim3 grid((A.width + 15) / 16, (A.height + 7) / 8, A.n_poses);
    raycast_backward_kernel<<<grid, 128, 0, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    pose_sum_kernel<<<A.n_poses, 256, 0, s>>>(A.partial, (int)(grid.x * grid.y), A.grad_pose);
    return cudaGetLastError();
}

}  // namespace mv
