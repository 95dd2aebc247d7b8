// mv_track.cu -- depth-map conversion and point-to-plane ICP (sm_103a).
//
// Sec. Depth Map Conversion: every pixel's vertex v = K^-1 [x, y, 1]^T D(x, y)
// and the normal (v(x+1, y) - v(x, y)) x (v(x, y+1) - v(x, y)), here
// normalised and turned to face the camera; Sec. Camera Tracking: the pose
// that aligns these vertices with the model maps of the previous raycast, by
// iterated point-to-plane ICP with projective data association.
//
// One linearisation is one kernel: every pixel of the current frame is moved
// by the current estimate, projected into the model's camera, associated with
// the model vertex / normal at the nearest pixel (rejected beyond a distance
// or normal-angle threshold), and contributes J^T J, J^T r, r^2 and a count
// (29 values) to a per-CTA partial (lanes and warps in FP32, the CTA's 8
// warp sums and everything after in FP64).  mv_icp_linearize adds the
// partials on the host in a fixed order; mv_track keeps the whole Gauss-Newton
// loop on the device: the pose lives in device memory, and the last CTA of
// each linearisation adds the partials in a fixed order, solves the 6x6
// system and updates the pose, so the iterations run back to back with no
// host round trip.
#include "mv_internal.cuh"

namespace mv {

struct Mat34f {
    float r[9];  // row-major rotation
    float t[3];
};

__global__ void __launch_bounds__(256) depth_maps_kernel(const float *__restrict__ depth, int W, int H, float fx,
                                                         float fy, float cx, float cy, float z_min, float z_max,
                                                         Mat34f T, float *__restrict__ vertex,
                                                         float *__restrict__ normal)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W * H) return;
    const int x = p % W, y = p / W;
    auto valid = [&](float D) { return D > 0.f && D >= z_min && D <= z_max; };
    auto backproject = [&](int xx, int yy, float D, float v[3]) {
        v[0] = ((float)xx - cx) / fx * D;
        v[1] = ((float)yy - cy) / fy * D;
        v[2] = D;
    };
    const float D = __ldg(depth + p);
    float v[3] = {0.f, 0.f, 0.f}, n[3] = {0.f, 0.f, 0.f};
    if (valid(D)) {
        backproject(x, y, D, v);
        if (x + 1 < W && y + 1 < H) {
            const float Dx = __ldg(depth + p + 1), Dy = __ldg(depth + p + W);
            if (valid(Dx) && valid(Dy)) {
                float vx[3], vy[3];
                backproject(x + 1, y, Dx, vx);
                backproject(x, y + 1, Dy, vy);
                const float a0 = vx[0] - v[0], a1 = vx[1] - v[1], a2 = vx[2] - v[2];
                const float b0 = vy[0] - v[0], b1 = vy[1] - v[1], b2 = vy[2] - v[2];
                float c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
                const float len = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
                if (len > 0.f) {
                    // face the camera (the side the raycast normals face)
                    const float sgn = (c0 * v[0] + c1 * v[1] + c2 * v[2] > 0.f) ? -1.f : 1.f;
                    n[0] = sgn * c0 / len;
                    n[1] = sgn * c1 / len;
                    n[2] = sgn * c2 / len;
                }
            }
        }
    }
    float vo[3] = {0.f, 0.f, 0.f}, no[3] = {0.f, 0.f, 0.f};
    if (valid(D)) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            vo[a] = T.r[3 * a] * v[0] + T.r[3 * a + 1] * v[1] + T.r[3 * a + 2] * v[2] + T.t[a];
            no[a] = T.r[3 * a] * n[0] + T.r[3 * a + 1] * n[1] + T.r[3 * a + 2] * n[2];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vertex[3 * (size_t)p + a] = vo[a];
        normal[3 * (size_t)p + a] = no[a];
    }
}

cudaError_t launch_depth_maps(const float *depth, const mv_intrinsics &K, float z_min, float z_max,
                              const double *T, float *vertex, float *normal, cudaStream_t s)
{
    Mat34f M;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) M.r[3 * a + b] = T ? (float)T[4 * a + b] : (a == b ? 1.f : 0.f);
        M.t[a] = T ? (float)T[4 * a + 3] : 0.f;
    }
    const int n = K.width * K.height;
    depth_maps_kernel<<<(n + 255) / 256, 256, 0, s>>>(depth, K.width, K.height, K.fx, K.fy, K.cx, K.cy, z_min,
                                                      z_max, M, vertex, normal);
    return cudaGetLastError();
}

constexpr int kIcpTerms = 29;  // 21 of J^T J (upper triangle, row-major), 6 of J^T r, r^2, count

struct IcpArgs {
    const float *vertex;   // current frame, camera frame
    const float *normal;
    int W, H;
    Mat34f est;            // current estimate, camera to world
    const float *mvertex;  // model maps (world frame), same size as the frame
    const float *mnormal;
    Mat34f model_inv;      // world to model camera
    float fx, fy, cx, cy;
    float dist2, cos_min;
    float *partials;       // gridDim.x x kIcpTerms
};

// Device state of mv_track's Gauss-Newton loop.
struct IcpLoop {
    double *T;      // current estimate, camera to world (row-major 4x4)
    double *sys;    // the last linearisation: A (36), b (6), r^2, count
    int *state;     // [0] stopped (too few inliers or a failed solve), [1] CTAs done
};

// 1 / sqrt(d) for d > 0: a float seed refined by one Newton step
// y <- y (3 - d y^2) / 2 in FP64 (the relative error e becomes about 1.5 e^2:
// from the seed's few 1e-7 to about 1e-13, far below what a Gauss-Newton
// increment needs) -- a short dependent chain where FP64 sqrt and division
// are long ones on B300.
__device__ __forceinline__ double inv_sqrt(double d)
{
    if (d > 1e-30 && d < 1e30) {
        const double y = (double)rsqrtf((float)d);
        return y * (1.5 - 0.5 * d * y * y);
    }
    return 1.0 / sqrt(d);
}

// The coefficients of the twist's exponential at q = th^2 = |phi|^2:
// sin(th)/th, (1 - cos th)/th^2, (th - sin th)/th^3.  For th < 0.1 rad (the
// Gauss-Newton increments of tracking) from the Maclaurin series in th^2,
// nested by the ratio of consecutive terms; the first omitted term
// (th^10 / 11!, / 12!, / 13!) is below 3e-18 relative, so the series is exact
// in double.  Every lane computes all three (no divergence).
__device__ __forceinline__ void twist_coefs(double q, double &a, double &b, double &c)
{
    if (q < 1e-2) {
        a = 1.0 - q * (1.0 / 6) * (1.0 - q * (1.0 / 20) * (1.0 - q * (1.0 / 42) * (1.0 - q * (1.0 / 72))));
        b = 0.5 * (1.0 - q * (1.0 / 12) * (1.0 - q * (1.0 / 30) * (1.0 - q * (1.0 / 56) * (1.0 - q * (1.0 / 90)))));
        c = (1.0 / 6) * (1.0 - q * (1.0 / 20) * (1.0 - q * (1.0 / 42) * (1.0 - q * (1.0 / 72) * (1.0 - q * (1.0 / 110)))));
        return;
    }
    const double th = sqrt(q), sn = sin(th);
    a = sn / th;
    b = (1.0 - cos(th)) / q;
    c = (th - sn) / (q * th);
}

// Warp 0 of the last CTA: the Gauss-Newton step from the 29 sums.  The
// 6x6 system is reported as summed; A x = b is solved by a right-looking
// Cholesky factorisation (per column one reciprocal square root, then the
// column and the trailing triangle updated one entry per lane) and two
// column-oriented triangular solves; then T <- exp(x^) T (Rodrigues, the
// 3x3 products one entry per lane).  The loop stops (state[0]) when fewer
// than 6 pixels associate or a pivot is not positive.
__device__ __forceinline__ void icp_step_warp(const double *tot, const IcpLoop &L)
{
    __shared__ double sA[36], sy[6], sinv[6], sP[9], sR[9], sV[9], st[3], sT[16];
    __shared__ int s_fail;
    const int lane = threadIdx.x;
    if (lane < 21) {  // upper-triangle sums, row-major -> both triangles
        int i = 0, r = lane;
        while (r >= 6 - i) { r -= 6 - i; ++i; }
        sA[6 * i + i + r] = sA[6 * (i + r) + i] = tot[lane];
    }
    if (lane < 6) sy[lane] = tot[21 + lane];
    if (lane == 0) s_fail = __double2ll_rn(tot[28]) < 6;
    __syncwarp();
    for (int e = lane; e < 36; e += 32) L.sys[e] = sA[e];
    if (lane < 6) L.sys[36 + lane] = sy[lane];
    if (lane == 0) {
        L.sys[42] = tot[27];
        L.sys[43] = tot[28];
        L.state[1] = 0;  // for the next linearisation, which starts after this kernel
    }
    for (int j = 0; j < 6; ++j) {
        __syncwarp();
        if (s_fail) break;
        if (lane == 0) {
            const double d = sA[7 * j];
            if (d > 0.0) sinv[j] = inv_sqrt(d);
            else s_fail = 1;
        }
        __syncwarp();
        if (s_fail) break;
        if (lane > j && lane < 6) sA[6 * lane + j] *= sinv[j];  // L_ij
        __syncwarp();
        const int m = 5 - j;  // trailing lower triangle: rows and columns j+1 .. 5
        if (lane < m * (m + 1) / 2) {
            int i = 0, r = lane;
            while (r > i) { r -= i + 1; ++i; }
            const int row = j + 1 + i, col = j + 1 + r;
            sA[6 * row + col] -= sA[6 * row + j] * sA[6 * col + j];
        }
    }
    __syncwarp();
    if (s_fail) {
        if (lane == 0) L.state[0] = 1;
        return;
    }
    for (int j = 0; j < 6; ++j) {  // L y = b
        if (lane == 0) sy[j] *= sinv[j];
        __syncwarp();
        if (lane > j && lane < 6) sy[lane] -= sA[6 * lane + j] * sy[j];
        __syncwarp();
    }
    for (int j = 5; j >= 0; --j) {  // L^T x = y
        if (lane == 0) sy[j] *= sinv[j];
        __syncwarp();
        if (lane < j) sy[lane] -= sA[6 * j + lane] * sy[j];
        __syncwarp();
    }
    // x = (rho, phi) = sy: T <- exp(x^) T
    const double p0 = sy[3], p1 = sy[4], p2 = sy[5];
    double ca, cb, cc;
    twist_coefs(p0 * p0 + p1 * p1 + p2 * p2, ca, cb, cc);
    if (lane < 9) {
        const double P[9] = {0.0, -p2, p1, p2, 0.0, -p0, -p1, p0, 0.0};
        sP[lane] = P[lane];
    }
    if (lane < 16) sT[lane] = L.T[lane];
    __syncwarp();
    if (lane < 9) {
        const int i = lane / 3, k = lane % 3;
        const double P2 = sP[3 * i] * sP[k] + sP[3 * i + 1] * sP[3 + k] + sP[3 * i + 2] * sP[6 + k];
        const double I = i == k ? 1.0 : 0.0;
        sR[lane] = I + ca * sP[lane] + cb * P2;
        sV[lane] = I + cb * sP[lane] + cc * P2;
    }
    __syncwarp();
    if (lane < 3) st[lane] = sV[3 * lane] * sy[0] + sV[3 * lane + 1] * sy[1] + sV[3 * lane + 2] * sy[2];
    __syncwarp();
    if (lane < 12) {
        const int i = lane >> 2, c = lane & 3;
        double acc = sR[3 * i] * sT[c] + sR[3 * i + 1] * sT[4 + c] + sR[3 * i + 2] * sT[8 + c];
        if (c == 3) acc += st[i];
        L.T[lane] = acc;
    } else if (lane < 16) {
        L.T[lane] = lane == 15 ? 1.0 : 0.0;
    }
}

// hi + lo += x, with the rounding error of hi + x kept in lo (Knuth's
// TwoSum: s = hi + x, b = s - hi, error (hi - (s - b)) + (x - b), exact in
// round-to-nearest), so that hi + lo carries about twice FP32's precision.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x)
{
    const float s = __fadd_rn(hi, x);
    const float b = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, b)), __fsub_rn(x, b));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// One CTA of kIcpCta threads per SM: the partials the last CTA of a device
// step adds are as few as the SMs, each term's added by kIcpSplit threads.
constexpr int kIcpCta = 512;
constexpr int kIcpSplit = 16;
static_assert(kIcpSplit * kIcpTerms <= kIcpCta, "ICP partial split");

// LOOP: the estimate is read from L.T, nothing runs once the loop stopped,
// and the last CTA to finish completes the Gauss-Newton step.
template <bool LOOP>
__global__ void __launch_bounds__(kIcpCta) icp_system_kernel(IcpArgs A, IcpLoop L)
{
    if (LOOP) {
        if (*(volatile int *)L.state) return;  // written by an earlier launch
        __shared__ float s_est[12];
        if (threadIdx.x < 12) {
            const int a = threadIdx.x < 9 ? threadIdx.x / 3 : threadIdx.x - 9;
            const int b = threadIdx.x < 9 ? threadIdx.x % 3 : 3;
            s_est[threadIdx.x] = (float)L.T[4 * a + b];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 9; ++k) A.est.r[k] = s_est[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) A.est.t[k] = s_est[9 + k];
    }
    float acc[kIcpTerms];
#pragma unroll
    for (int k = 0; k < kIcpTerms; ++k) acc[k] = 0.f;
    const int n = A.W * A.H;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float nl0 = A.normal[3 * p], nl1 = A.normal[3 * p + 1], nl2 = A.normal[3 * p + 2];
        if (nl0 == 0.f && nl1 == 0.f && nl2 == 0.f) continue;
        const float vl0 = A.vertex[3 * p], vl1 = A.vertex[3 * p + 1], vl2 = A.vertex[3 * p + 2];
        float v[3], nn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[a] = A.est.r[3 * a] * vl0 + A.est.r[3 * a + 1] * vl1 + A.est.r[3 * a + 2] * vl2 + A.est.t[a];
            nn[a] = A.est.r[3 * a] * nl0 + A.est.r[3 * a + 1] * nl1 + A.est.r[3 * a + 2] * nl2;
        }
        float q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            q[a] = A.model_inv.r[3 * a] * v[0] + A.model_inv.r[3 * a + 1] * v[1] + A.model_inv.r[3 * a + 2] * v[2] +
                   A.model_inv.t[a];
        if (!(q[2] > 0.f)) continue;
        const float u = A.fx * q[0] / q[2] + A.cx, w = A.fy * q[1] / q[2] + A.cy;
        const int ui = (int)floorf(u + 0.5f), wi = (int)floorf(w + 0.5f);
        if (ui < 0 || wi < 0 || ui >= A.W || wi >= A.H) continue;
        const size_t m = (size_t)wi * A.W + ui;
        const float N0 = A.mnormal[3 * m], N1 = A.mnormal[3 * m + 1], N2 = A.mnormal[3 * m + 2];
        if (!(N0 * N0 + N1 * N1 + N2 * N2 > 0.25f)) continue;  // model miss (normal 0)
        const float V0 = A.mvertex[3 * m], V1 = A.mvertex[3 * m + 1], V2 = A.mvertex[3 * m + 2];
        const float d0 = V0 - v[0], d1 = V1 - v[1], d2 = V2 - v[2];
        if (!(d0 * d0 + d1 * d1 + d2 * d2 <= A.dist2)) continue;
        if (!(nn[0] * N0 + nn[1] * N1 + nn[2] * N2 >= A.cos_min)) continue;
        const float r = N0 * d0 + N1 * d1 + N2 * d2;
        // x = (rho, phi): v -> v + rho + phi x v, so dr/dx = -[N, v x N]
        const float J[6] = {N0, N1, N2, v[1] * N2 - v[2] * N1, v[2] * N0 - v[0] * N2, v[0] * N1 - v[1] * N0};
        int k = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = i; j < 6; ++j) acc[k++] += J[i] * J[j];
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[21 + i] += J[i] * r;
        acc[27] += r * r;
        acc[28] += 1.f;
    }
    // CTA sum: each warp by a pairwise tree of FP32 shuffles, then the CTA's
    // warps by a pairwise tree in FP32 (9 roundings on top of the lanes' own
    // sums).  B300 runs FP64 at a small fraction of its FP32 rate, and a
    // warp's FP64 instruction holds that pipe however few lanes it has: an
    // FP64 shuffle tree took about half the kernel's time, and the per-warp
    // FP64 conversions and FP64 sum of the warps' results a tenth (a device
    // step 27.0 -> 24.3 us without them).
    constexpr int kWarps = kIcpCta / 32;
    __shared__ float s_part[kWarps][kIcpTerms];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kIcpTerms; ++k) {
        float x = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) s_part[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kIcpTerms) {
        float v[kWarps];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) v[w] = s_part[w][threadIdx.x];
#pragma unroll
        for (int h = kWarps / 2; h > 0; h >>= 1)
#pragma unroll
            for (int w = 0; w < h; ++w) v[w] += v[w + h];
        A.partials[(size_t)blockIdx.x * kIcpTerms + threadIdx.x] = v[0];
    }
    if (!LOOP) return;
    // the last CTA to finish adds the partials (kIcpSplit threads per term,
    // each a fixed stride of CTAs, then those sums in order: a fixed order)
    // by compensated FP32 summation (about 48 bits for these few terms, at
    // FP32 speed), solves and updates the estimate
    __shared__ bool s_last;
    __shared__ float s_hi[kIcpTerms][kIcpSplit], s_lo[kIcpTerms][kIcpSplit];
    __shared__ double s_tot[kIcpTerms];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&L.state[1], 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < kIcpSplit * kIcpTerms) {
        const int k = threadIdx.x / kIcpSplit, j = threadIdx.x % kIcpSplit, G = (int)gridDim.x;
        const float *pk = A.partials + k;
        float hi = 0.f, lo = 0.f;
        int g = j;
        for (; g + 7 * kIcpSplit < G; g += 8 * kIcpSplit) {  // 8 loads in flight, added in the same order
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(pk + (size_t)(g + kIcpSplit * u) * kIcpTerms);
#pragma unroll
            for (int u = 0; u < 8; ++u) two_sum_add(hi, lo, v[u]);
        }
        for (; g < G; g += kIcpSplit) two_sum_add(hi, lo, __ldcg(pk + (size_t)g * kIcpTerms));
        s_hi[k][j] = hi;
        s_lo[k][j] = lo;
    }
    __syncthreads();
    if (threadIdx.x < kIcpTerms) {
        float hi = 0.f, lo = 0.f;
        for (int j = 0; j < kIcpSplit; ++j) {
            two_sum_add(hi, lo, s_hi[threadIdx.x][j]);
            lo += s_lo[threadIdx.x][j];
        }
        s_tot[threadIdx.x] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    icp_step_warp(s_tot, L);
}

int icp_grid(int num_sms) { return num_sms; }

static IcpArgs icp_args(const float *vertex, const float *normal, const mv_intrinsics &K, const double *T_est,
                        const float *mvertex, const float *mnormal, const double *T_model, float dist,
                        float cos_min, float *partials)
{
    IcpArgs A;
    A.vertex = vertex;
    A.normal = normal;
    A.W = K.width;
    A.H = K.height;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            A.est.r[3 * a + b] = T_est ? (float)T_est[4 * a + b] : 0.f;
            A.model_inv.r[3 * a + b] = (float)T_model[4 * b + a];  // R^T
        }
        A.est.t[a] = T_est ? (float)T_est[4 * a + 3] : 0.f;
    }
    for (int a = 0; a < 3; ++a) {  // -R^T t in FP64, then rounded
        double x = 0.0;
        for (int b = 0; b < 3; ++b) x -= T_model[4 * b + a] * T_model[4 * b + 3];
        A.model_inv.t[a] = (float)x;
    }
    A.mvertex = mvertex;
    A.mnormal = mnormal;
    A.fx = K.fx;
    A.fy = K.fy;
    A.cx = K.cx;
    A.cy = K.cy;
    A.dist2 = dist * dist;
    A.cos_min = cos_min;
    A.partials = partials;
    return A;
}

cudaError_t launch_icp_system(const float *vertex, const float *normal, const mv_intrinsics &K,
                              const double *T_est, const float *mvertex, const float *mnormal,
                              const double *T_model, float dist, float cos_min, float *partials, int grid,
                              cudaStream_t s)
{
    const IcpArgs A = icp_args(vertex, normal, K, T_est, mvertex, mnormal, T_model, dist, cos_min, partials);
    icp_system_kernel<false><<<grid, kIcpCta, 0, s>>>(A, IcpLoop{nullptr, nullptr, nullptr});
    return cudaGetLastError();
}

// One Gauss-Newton step of mv_track on the device (estimate in T_dev; loop
// state: 16 doubles of pose, 44 of system, 2 ints).
cudaError_t launch_icp_step(const float *vertex, const float *normal, const mv_intrinsics &K, double *T_dev,
                            double *sys_dev, int *state_dev, const float *mvertex, const float *mnormal,
                            const double *T_model, float dist, float cos_min, float *partials, int grid,
                            cudaStream_t s)
{
    const IcpArgs A = icp_args(vertex, normal, K, nullptr, mvertex, mnormal, T_model, dist, cos_min, partials);
    icp_system_kernel<true><<<grid, kIcpCta, 0, s>>>(A, IcpLoop{T_dev, sys_dev, state_dev});
    return cudaGetLastError();
}

}  // namespace mv
