// mv_extract.cu -- surface points of one volume (sm_103a).
//
// The point cloud that stands for a volume once it leaves the map (Sec.
// Insertion and Removal); the number of points is the paper's resolution
// measure (Table 1, vertices).  One point per edge between 6-neighbour voxels
// i and i + e_a that are both observed and lie on different sides of the
// surface, at the zero of the linear interpolation along the edge.
//
// A persistent grid walks the bricks; a brick is skipped whole when it holds
// no observed voxel (kFlagEmpty) or when its cell-brick flag says that it and
// its +x/+y/+z neighbours hold no observed F <= 0 voxel (no edge can cross).
// Each CTA handles one brick at a time, 4 voxels per thread; points are
// appended with one atomic per warp.
#include "mv_internal.cuh"

namespace mv {

struct ExtractOut {
    float *xyz;              // 3 per point, or null
    uint8_t *rgb;            // 3 per point, or null
    unsigned long long *edge;  // 1 per point, or null
    unsigned long long cap;
    unsigned long long *count;
};

template <int FMT>
__device__ __forceinline__ void load_fw(const VolDev &v, long long off, float &F, float &W)
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

// round half up of a non-negative value
__device__ __forceinline__ uint32_t round_half_up(float x)
{
    return (uint32_t)floorf(x + 0.5f);
}

template <int FMT>
__device__ void extract_brick(const VolDev &v, int bx, int by, int bz, const ExtractOut &o)
{
    const int t = threadIdx.x;
    const int lx0 = (t & 1) * 4, ly = (t >> 1) & 7, lz = t >> 4;
    const int gy = by * kBrick + ly, gz = bz * kBrick + lz;
    float px[12], py[12], pz[12];
    uint32_t col[12];
    unsigned long long eid[12];
    int n = 0;
    if (gy < v.r[1] && gz < v.r[2]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gx = bx * kBrick + lx0 + j;
            if (gx >= v.r[0]) break;
            const long long off = vox_offset(v, gx, gy, gz);
            float F0, W0;
            load_fw<FMT>(v, off, F0, W0);
            if (!(W0 > 0.f)) continue;
            const uint32_t c0 = __ldg(v.rgba + off);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int nx = gx + (a == 0), ny = gy + (a == 1), nz = gz + (a == 2);
                if (nx >= v.r[0] || ny >= v.r[1] || nz >= v.r[2]) continue;
                const long long off1 = vox_offset(v, nx, ny, nz);
                float F1, W1;
                load_fw<FMT>(v, off1, F1, W1);
                if (!(W1 > 0.f) || ((F0 > 0.f) == (F1 > 0.f))) continue;
                const float tt = F0 / (F0 - F1);
                px[n] = ((float)(v.h[0] + gx) + (a == 0 ? tt : 0.f)) * v.s;
                py[n] = ((float)(v.h[1] + gy) + (a == 1 ? tt : 0.f)) * v.s;
                pz[n] = ((float)(v.h[2] + gz) + (a == 2 ? tt : 0.f)) * v.s;
                const uint32_t c1 = __ldg(v.rgba + off1);
                uint32_t cc = 0u;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float a0 = (float)((c0 >> (8 * ch)) & 0xFFu), a1 = (float)((c1 >> (8 * ch)) & 0xFFu);
                    cc |= min(255u, round_half_up(fmaf(tt, a1 - a0, a0))) << (8 * ch);
                }
                col[n] = cc;
                eid[n] = 3ull * (((unsigned long long)gz * v.r[1] + gy) * v.r[0] + gx) + a;
                ++n;
            }
        }
    }
    // one atomic per warp
    const int lane = t & 31;
    int incl = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(o.count, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31) + (unsigned long long)(incl - n);
    for (int k = 0; k < n; ++k) {
        const unsigned long long i = base + k;
        if (i >= o.cap) break;
        if (o.xyz) {
            o.xyz[3 * i] = px[k];
            o.xyz[3 * i + 1] = py[k];
            o.xyz[3 * i + 2] = pz[k];
        }
        if (o.rgb) {
            o.rgb[3 * i] = (uint8_t)(col[k] & 0xFFu);
            o.rgb[3 * i + 1] = (uint8_t)((col[k] >> 8) & 0xFFu);
            o.rgb[3 * i + 2] = (uint8_t)((col[k] >> 16) & 0xFFu);
        }
        if (o.edge) o.edge[i] = eid[k];
    }
}

__global__ void __launch_bounds__(128) extract_kernel(VolDev v, ExtractOut o)
{
    for (long long b = blockIdx.x; b < v.nbricks; b += gridDim.x) {
        const uint8_t bf = __ldg(v.bflag + b);
        if (bf & kFlagEmpty) continue;                           // nothing observed
        if (v.cflag && (__ldg(v.cflag + b) & kCellSkip)) continue;  // no observed F <= 0 nearby
        const int bx = (int)(b % v.nb[0]);
        const int by = (int)((b / v.nb[0]) % v.nb[1]);
        const int bz = (int)(b / ((long long)v.nb[0] * v.nb[1]));
        switch (v.fmt) {
        case MV_TSDF_F32: extract_brick<MV_TSDF_F32>(v, bx, by, bz, o); break;
        case MV_TSDF_F16: extract_brick<MV_TSDF_F16>(v, bx, by, bz, o); break;
        default: extract_brick<MV_TSDF_I16>(v, bx, by, bz, o); break;
        }
    }
}

cudaError_t launch_extract(const VolDev &v, float *xyz, uint8_t *rgb, unsigned long long *edge,
                           unsigned long long cap, unsigned long long *count, int num_sms, cudaStream_t s)
{
    ExtractOut o{xyz, rgb, edge, cap, count};
    long long blocks = v.nbricks;
    const long long most = (long long)num_sms * 8;
    if (blocks > most) blocks = most;
    if (blocks < 1) blocks = 1;
    extract_kernel<<<(unsigned)blocks, 128, 0, s>>>(v, o);
    return cudaGetLastError();
}

// A box of a volume's voxels in linear order (x fastest), gathered from the
// brick-major storage: voxels lo .. lo + n - 1 per axis.
template <typename T>
__global__ void __launch_bounds__(256) gather_box_kernel(const T *__restrict__ src, int nb0, int nb1, int lo0,
                                                         int lo1, int lo2, int n0, int n1, long long total,
                                                         T *__restrict__ dst)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % n0) + lo0;
        const int y = (int)((i / n0) % n1) + lo1;
        const int z = (int)(i / ((long long)n0 * n1)) + lo2;
        const long long b = ((long long)(z >> 3) * nb1 + (y >> 3)) * nb0 + (x >> 3);
        dst[i] = src[b * kBrickVox + (((z & 7) << 6) | ((y & 7) << 3) | (x & 7))];
    }
}

cudaError_t launch_gather_box(const void *src, int elem_bytes, const int nb[3], const int lo[3], const int n[3],
                              void *dst, int num_sms, cudaStream_t s)
{
    const long long total = (long long)n[0] * n[1] * n[2];
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
    if (blocks < 1) blocks = 1;
    if (elem_bytes == 8)
        gather_box_kernel<unsigned long long><<<(unsigned)blocks, 256, 0, s>>>(
            static_cast<const unsigned long long *>(src), nb[0], nb[1], lo[0], lo[1], lo[2], n[0], n[1], total,
            static_cast<unsigned long long *>(dst));
    else
        gather_box_kernel<unsigned><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const unsigned *>(src), nb[0], nb[1],
                                                                    lo[0], lo[1], lo[2], n[0], n[1], total,
                                                                    static_cast<unsigned *>(dst));
    return cudaGetLastError();
}

}  // namespace mv
