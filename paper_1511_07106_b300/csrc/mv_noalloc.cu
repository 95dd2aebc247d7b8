// mv_noalloc.cu -- mv_integrate_noalloc: frame integration into a caller-owned
// volume without any allocation (see include/mvtsdf.h).
//
// For callers that cannot allocate GPU memory: the brick work list and the
// per-call constants live in one fixed, file-scope device array instead of
// context-owned buffers.  The kernels are the same ones mv_integrate uses.
#include <mutex>

#include "mv_internal.cuh"

namespace mv {
cudaError_t launch_frame_setup(const VolDev *, int, const FrameParams &, VolFrame *, unsigned *, cudaStream_t,
                               VisList *);
cudaError_t launch_brick_list(const VolDev *, int, const VolFrame *, const FrameParams &, long long,
                              long long, uint2 *, unsigned *, int, cudaStream_t, const VisList *,
                              const unsigned *, const unsigned *, uint2 *, long long);
cudaError_t launch_depth_max(const float *, const FrameParams &, unsigned *, int, cudaStream_t, unsigned *);
cudaError_t launch_integrate(const VolDev *, const VolFrame *, const uint2 *, const unsigned *,
                             const FrameParams &, const float *, const uint8_t *, Stats *, int,
                             cudaStream_t, uint2 *, unsigned *, unsigned);
int integrate_occupancy_grid(int num_sms);
bool valid_config(const mv_config &c);
}  // namespace mv

using namespace mv;

namespace {

// working array layout: [brick list | volume descriptor | camera constants | counter]
constexpr size_t kListBytes = (size_t)MV_NOALLOC_MAX_BRICKS * sizeof(uint2);
constexpr size_t kVolOff = kListBytes;
constexpr size_t kFrameOff = kVolOff + 256;
constexpr size_t kCounterOff = kFrameOff + 256;
constexpr size_t kScratchBytes = kCounterOff + 256;
static_assert(sizeof(VolDev) <= 256 && sizeof(VolFrame) <= 256, "scratch slots too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Per-device address of g_noalloc_scratch, SM count and integration grid.
// In host code the symbol's name is only a host-side stand-in, never a device
// address: a kernel must be given the address that cudaGetSymbolAddress
// returns for the current device.  The address belongs to the module loaded
// in the device's current context; a device reset (cudaDeviceReset) or a new
// primary context loads the module again, possibly elsewhere.  So every call
// whose stream is not being captured looks the address up again (cheap once
// the module is loaded) and refreshes the cache; a call on a capturing
// stream, where that lookup could be refused, uses the cached address of the
// device's last uncaptured call.  The SM count and the grid depend only on
// the device and are kept from the first call.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
int g_grid[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

cudaError_t device_scratch(int dev, cudaStream_t s, unsigned char **ptr, int *grid, int *sms)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_sms[dev]) {
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_grid[dev] = integrate_occupancy_grid(n);
        g_sms[dev] = n;
    }
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    } else if (!g_scratch_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;  // no uncaptured call has looked it up yet
    }
    *ptr = g_scratch_ptr[dev];
    *grid = g_grid[dev];
    *sms = g_sms[dev];
    return cudaSuccess;
}

// Stores the caller's volume descriptor into the working array (a kernel
// parameter, so no host-to-device copy is needed).
__global__ void store_voldev_kernel(VolDev v, VolDev *dst)
{
    if (threadIdx.x == 0) *dst = v;
}

bool is_finite(double x) { return x == x && x - x == 0.0; }

}  // namespace

extern "C" mv_status mv_integrate_noalloc(const mv_volume_view *vol, const mv_config *cfg,
                                          const float *depth, const uint8_t *rgb,
                                          const mv_intrinsics *K, const double T[16], void *stream)
{
    if (!vol || !depth || !K || !T || !vol->fw || !vol->rgba || !vol->brick_flags) return MV_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(vol->fw) & 15u) || (reinterpret_cast<uintptr_t>(vol->rgba) & 15u))
        return MV_ERR_ARG;
    if (!aligned_to({depth}, 4)) return MV_ERR_ARG;
    mv_config c;
    if (cfg) {
        c = *cfg;
    } else {
        mv_config_default(&c);
    }
    if (!valid_config(c)) return MV_ERR_ARG;
    const mv_volume_desc &d = vol->desc;
    if (d.fmt < MV_TSDF_F32 || d.fmt > MV_TSDF_I16 || !(d.voxel_size > 0.f) || !is_finite(d.voxel_size))
        return MV_ERR_ARG;
    if (d.fmt != MV_TSDF_F32 && c.w_max > 65535.f) return MV_ERR_ARG;
    long long nbricks = 1;
    int nb[3];
    for (int a = 0; a < 3; ++a) {
        if (d.h_r[a] < 2 || d.h_r[a] > 8192) return MV_ERR_ARG;
        nb[a] = (d.h_r[a] + kBrick - 1) / kBrick;
        nbricks *= nb[a];
    }
    if (nbricks > MV_NOALLOC_MAX_BRICKS) return MV_ERR_CAPACITY;
    if (K->width <= 0 || K->height <= 0 || K->width > 16384 || K->height > 16384 || !(K->fx > 0.f) ||
        !(K->fy > 0.f) || !is_finite(K->fx) || !is_finite(K->fy) || !is_finite(K->cx) || !is_finite(K->cy))
        return MV_ERR_ARG;
    for (int i = 0; i < 16; ++i)
        if (!is_finite(T[i])) return MV_ERR_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MV_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *scratch = nullptr;
    int grid = 0, sms = 0;
    if (device_scratch(dev, s, &scratch, &grid, &sms) != cudaSuccess) return MV_ERR_CUDA;
    uint2 *list = reinterpret_cast<uint2 *>(scratch);
    VolDev *vdev = reinterpret_cast<VolDev *>(scratch + kVolOff);
    VolFrame *vframe = reinterpret_cast<VolFrame *>(scratch + kFrameOff);
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + kCounterOff);

    VolDev v{};
    v.fw = vol->fw;
    v.rgba = reinterpret_cast<uint32_t *>(vol->rgba);
    v.bflag = vol->brick_flags;
    for (int a = 0; a < 3; ++a) {
        v.h[a] = d.h_t[a];
        v.r[a] = d.h_r[a];
        v.nb[a] = nb[a];
    }
    v.s = d.voxel_size;
    v.inv_s = 1.0f / d.voxel_size;
    v.fmt = d.fmt;
    v.id = 0;
    v.brick_base = 0;
    v.nbricks = nbricks;

    FrameParams P;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            P.R[3 * a + b] = T[4 * a + b];
            P.Rf[3 * a + b] = (float)T[4 * a + b];
        }
        P.t[a] = T[4 * a + 3];
        P.tf[a] = (float)T[4 * a + 3];
    }
    P.fx = K->fx; P.fy = K->fy; P.cx = K->cx; P.cy = K->cy;
    P.width = K->width; P.height = K->height;
    P.z_min = c.z_min; P.z_max = c.z_max;
    P.trunc_vox = c.trunc_voxels;
    P.w_max = c.w_max;
    P.color_w_max = c.color_w_max;
    P.ray_step = c.ray_step;
    P.n_bisect = c.n_bisect;

    store_voldev_kernel<<<1, 32, 0, s>>>(v, vdev);
    if (cudaGetLastError() != cudaSuccess) return MV_ERR_CUDA;
    // the frame setup zeroes the list counter and the depth maximum, the values
    // that must start at 0
    if (launch_frame_setup(vdev, 1, P, vframe, counter, s, nullptr) != cudaSuccess) return MV_ERR_CUDA;
    if (launch_depth_max(depth, P, counter + 1, sms, s, nullptr) != cudaSuccess) return MV_ERR_CUDA;
    if (launch_brick_list(vdev, 1, vframe, P, 0, nbricks, list, counter, sms, s, nullptr, counter + 1, nullptr,
                          nullptr, 0) !=
        cudaSuccess)
        return MV_ERR_CUDA;
    if (launch_integrate(vdev, vframe, list, counter, P, depth, rgb, nullptr, grid, s, nullptr, nullptr, 0u) != cudaSuccess)
        return MV_ERR_CUDA;
    return MV_OK;
}
