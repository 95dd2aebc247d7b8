// mv_merge.cu -- merge of raycast maps computed on different GPUs (sm_103a).
//
// Sec. Raycasting (last paragraph): every volume writes into one map and, per
// pixel, the hit with the shortest ray distance wins.  When the volumes of a
// frame are partitioned across GPUs (integration of different volumes is
// independent, Sec. Comparison to KinectFusion), each GPU raycasts its own
// volumes and the per-pixel winner is found by one all-reduce MIN over packed
// 64-bit keys (the bits of the ray distance tau above the global volume id:
// tau >= 0, so the bit order of the float is its numeric order, and equal
// distances go to the lower id, the single-GPU merge rule).  The winner's
// normal, colour and vertex then reach every GPU through an all-reduce SUM of
// the maps in which each GPU has cleared the pixels it did not win (x + 0 is
// exact, and exactly one GPU holds each hit).  The two kernels below are the
// per-pixel steps on either side of the first collective.
#include <float.h>

#include "mv_internal.cuh"

namespace mv {

constexpr long long kNoHit = 0x7FFFFFFFFFFFFFFFll;

__global__ void __launch_bounds__(256) pack_hits_kernel(const float *__restrict__ depth,
                                                        const int32_t *__restrict__ vol_id,
                                                        const int32_t *__restrict__ id_map, int32_t id_map_len,
                                                        long long n, long long *__restrict__ keys)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int id = vol_id[p];
        long long k = kNoHit;
        const float t = depth[p];
        if (id >= 0 && t > 0.f && t < FLT_MAX) {
            const int g = id_map ? (id < id_map_len ? id_map[id] : -1) : id;
            if (g >= 0) k = (long long)(((unsigned long long)__float_as_uint(t) << 32) | (unsigned)g);
        }
        keys[p] = k;
    }
}

__global__ void __launch_bounds__(256) merge_hits_kernel(const long long *__restrict__ best,
                                                         const long long *__restrict__ own,
                                                         long long n, float *__restrict__ depth,
                                                         int32_t *__restrict__ vol_id, float *__restrict__ normal,
                                                         uint32_t *__restrict__ rgba, float *__restrict__ vertex)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const long long b = best[p];
        const bool hit = b != kNoHit;
        if (depth) depth[p] = hit ? __uint_as_float((unsigned)((unsigned long long)b >> 32)) : 0.f;
        if (vol_id) vol_id[p] = hit ? (int32_t)(unsigned)((unsigned long long)b & 0xFFFFFFFFull) : -1;
        if (!hit || own[p] != b) {  // another GPU's volume (or none) won this pixel
            if (normal) normal[3 * p] = normal[3 * p + 1] = normal[3 * p + 2] = 0.f;
            if (rgba) rgba[p] = 0u;
            if (vertex) vertex[3 * p] = vertex[3 * p + 1] = vertex[3 * p + 2] = 0.f;
        }
    }
}

}  // namespace mv

using namespace mv;

namespace {

int grid_for(long long n)
{
    const long long b = (n + 255) / 256;
    return (int)(b < 148 * 8 ? (b > 0 ? b : 1) : 148 * 8);
}

}  // namespace

extern "C" mv_status mv_pack_hits(const float *depth, const int32_t *vol_id, const int32_t *id_map,
                                  int32_t id_map_len, int64_t n, int64_t *keys, void *stream)
{
    if (!depth || !vol_id || !keys || n < 0 || id_map_len < 0 || (id_map_len > 0 && !id_map)) return MV_ERR_ARG;
    if (!aligned_to({depth, vol_id, id_map}, 4) || !aligned_to({keys}, 8)) return MV_ERR_ARG;
    if (n == 0) return MV_OK;
    pack_hits_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
        depth, vol_id, id_map_len > 0 ? id_map : nullptr, id_map_len, n,
        reinterpret_cast<long long *>(keys));
    return cudaGetLastError() == cudaSuccess ? MV_OK : MV_ERR_CUDA;
}

extern "C" mv_status mv_merge_hits(const int64_t *best_keys, const int64_t *own_keys, int64_t n, float *depth,
                                   int32_t *vol_id, float *normal, uint8_t *rgba, float *vertex, void *stream)
{
    if (!best_keys || !own_keys || n < 0) return MV_ERR_ARG;
    if (!aligned_to({best_keys, own_keys}, 8) || !aligned_to({depth, vol_id, normal, rgba, vertex}, 4)) return MV_ERR_ARG;
    if (n == 0) return MV_OK;
    merge_hits_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const long long *>(best_keys), reinterpret_cast<const long long *>(own_keys),
        n, depth, vol_id, normal, reinterpret_cast<uint32_t *>(rgba), vertex);
    return cudaGetLastError() == cudaSuccess ? MV_OK : MV_ERR_CUDA;
}
