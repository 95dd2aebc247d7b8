// mv_internal.cuh -- device-side data structures shared by the kernels and the
// runtime of the multi-volume TSDF library (sm_103a).
//
// Volume storage is brick-major: a volume of h_r voxels per axis is padded to
// whole 8x8x8 bricks; brick (bx, by, bz) is stored contiguously at brick index
// (bz * nby + by) * nbx + bx, and inside a brick voxel (lx, ly, lz) sits at
// (lz * 8 + ly) * 8 + lx.  Padding voxels (index >= h_r) are never integrated
// and keep W = 0.  Every brick also has one flag byte summarising its voxels
// (all observed and positive / all unobserved / no observed voxel with F <= 0),
// maintained by the integration kernel, and every brick has one "cell brick"
// byte saying whether the trilinear cells whose lower corner lies in the brick
// can be stepped over by the raycast (see mv_raycast.cu).  Both byte arrays
// live in one allocation: voxel-brick flags first, then cell-brick flags.
//
// Resident volumes also carry per-voxel and per-cell bit masks (derived data,
// rebuilt from the voxels after a host write or a swap-in, never swapped):
//   vmask, 16 x u64 per brick: rows [0, 8) = "observed" (W > 0) of slice z,
//          rows [8, 16) = "observed with stored F <= 0" of slice z; bit
//          8 y + x is voxel (x, y, z) of the brick;
//   cmask, 8 x (u64 V, u64 N) per brick: for the trilinear cell whose lower
//          corner is voxel (x, y, z) of the brick, bit 8 y + x of V is set when
//          all 8 corners are observed and of N when some corner is observed
//          with F <= 0 (corners beyond the brick come from its neighbours);
//   stamp, 1 x u32 per brick: the id of the last integration call whose work
//          list held the brick (lets the cell-mask refresh visit each cell
//          brick once).
// The raycast decides most samples from one 16-byte cmask load: a cell with
// N clear cannot end a bracket, and its V bit gives the march state.  With
// masks, a cell brick carries kCellSkip exactly when none of its cells has N
// set (a finer test than the brick summaries, which are used without masks).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>
#include <tuple>
#include <utility>

#include "mvtsdf.h"

namespace mv {

constexpr int kBrick = 8;
constexpr int kBrickVox = 512;
constexpr uint8_t kFlagFree = 1;   // every voxel of the brick has W > 0 and F > 0
constexpr uint8_t kFlagEmpty = 2;  // every voxel of the brick has W == 0
constexpr uint8_t kFlagNoNeg = 4;  // no voxel of the brick has W > 0 and F <= 0
constexpr uint8_t kFlagsNew = kFlagEmpty | kFlagNoNeg;  // a freshly cleared brick
// Cell-brick flag: no trilinear cell whose lower corner lies in the brick has
// an observed corner with F <= 0 (taken from the cell masks where the volume
// has them, else from the brick summaries: the 8 bricks b + {0,1}^3 all carry
// kFlagNoNeg, a stronger condition).
constexpr uint8_t kCellSkip = 1;
// Super brick: kSuper^3 cell bricks (32^3 voxels).  A super brick whose count
// of cell bricks without kCellSkip is 0 is crossed by the raycast in one step.
// Its 32-bit word holds that count in bits 0-7 (at most 64) and, for the
// super bricks within Chebyshev distance 1 (the 3^3 block around it, itself
// included, clipped to the grid) and 2 (the 5^3 block), how many have a
// non-zero count, in bits 8-15 (at most 27) and 16-23 (at most 125): with
// such a count 0 the raycast crosses the whole block in one step.
constexpr int kSuper = 4;
constexpr unsigned kSupCount = 0xFFu;
constexpr unsigned kSupNear1 = 1u << 8;
constexpr unsigned kSupNear2 = 1u << 16;
constexpr int kSupReach = 2;
constexpr int kMaxVolumes = 4096;

// One volume as the kernels see it.
struct VolDev {
    void *fw;          // brick-major TSDF+weight storage (8 B/voxel F32, 4 B/voxel F16/I16)
    uint32_t *rgba;    // brick-major RGBA8, A = colour weight
    uint8_t *bflag;    // one flag byte per brick
    uint8_t *cflag;    // one cell-brick byte per brick (may be null where no raycast reads it)
    unsigned *surf;    // bricks without kFlagNoNeg (0: no hit possible anywhere), may be null
    unsigned *sup;     // per super brick: counts of non-skippable cell bricks and neighbours (may be null)
    unsigned long long *vmask;  // per-voxel masks, 16 x u64 per brick (may be null)
    ulonglong2 *cmask;          // per-cell masks, 8 x (V, N) per brick (may be null)
    unsigned *stamp;            // per brick: id of the last integration that listed it (may be null)
    int h[3];          // lattice offset h_t
    int r[3];          // voxels per axis h_r
    int nb[3];         // bricks per axis
    int nsb[3];        // super bricks per axis, ceil(nb / kSuper)
    float s, inv_s;    // pitch and its reciprocal
    int fmt;           // mv_tsdf_fmt
    int id;            // public id (merge tie-break)
    long long brick_base;  // prefix sum of nbricks over the table (work-list indexing)
    long long nbricks;
};

// Camera position in one volume's global voxel units, split into an exact
// integer lattice part and a fraction in [0, 1): positions relative to the
// camera are then formed as (integer difference) - fraction in float32
// without losing the lattice alignment shared by volumes of equal pitch.
struct VolFrame {
    int cam_int[3];
    float cam_frac[3];
};

// Per-call parameters, passed by value.
struct FrameParams {
    double R[9];       // camera-to-world rotation, row-major
    double t[3];       // camera centre, metres
    float Rf[9];
    float tf[3];       // camera centre, metres, rounded to float (no FP64 in the kernels' per-pixel work)
    float fx, fy, cx, cy;
    int width, height;
    float z_min, z_max;
    float trunc_vox;
    float w_max;
    int color_w_max;
    float ray_step;
    int n_bisect;
};

// Volumes in the view of one call, nearest first (when there are at most
// kVisSortMax of them; table order otherwise), with prefix sums of their
// brick counts for the work-list kernel.  Built on the device by the per-call
// setup kernel.
constexpr int kVisSortMax = 256;
// Resident bricks from which the batched calls build their work list in two
// levels (super bricks in view, then their bricks).
constexpr long long kTwoLevelBricks = 1ll << 20;
// candidate volumes per raycast CTA held in shared memory
constexpr int kTileVolMax = 256;
struct VisList {
    int count;
    int pad;
    long long total;                  // bricks of the visible volumes
    long long stotal;                 // super bricks of the visible volumes
    int slot[kMaxVolumes];            // table slots
    long long base[kMaxVolumes + 1];  // prefix sums of nbricks over slot[]
    long long sbase[kMaxVolumes + 1]; // prefix sums of the super-brick counts over slot[]
};

// Flag allocation of a volume with nbricks bricks and nsuper super bricks:
// voxel-brick flags (1 B/brick), cell-brick flags (1 B/brick, 4-byte
// aligned so that a flag byte can be changed by a 32-bit atomic on its word),
// the count of bricks without kFlagNoNeg (u32, 8-byte aligned), then per
// super brick its word of counts (u32, see kSupCount).
inline size_t cflag_offset(long long nbricks) { return ((size_t)nbricks + 3) & ~(size_t)3; }
inline size_t flag_count_offset(long long nbricks)
{
    return (cflag_offset(nbricks) + (size_t)nbricks + 7) & ~(size_t)7;
}
inline size_t super_offset(long long nbricks) { return flag_count_offset(nbricks) + 8; }

// Device buffers that the kernels access as 4-byte words (floats, ints,
// packed colours) must start on a 4-byte boundary, 8-byte keys on an 8-byte
// one, or the access faults: the entry points refuse other pointers (null
// passes, for the optional ones) before any launch.
inline bool aligned_to(std::initializer_list<const void *> ps, uintptr_t a)
{
    for (const void *p : ps)
        if (reinterpret_cast<uintptr_t>(p) & (a - 1)) return false;
    return true;
}
inline size_t flag_alloc_bytes(long long nbricks, long long nsuper)
{
    return super_offset(nbricks) + 4 * (size_t)nsuper;
}

// Mask allocation of a volume: vmask (128 B per brick), cmask (128 B per
// brick), then the listing stamps (4 B per brick).
constexpr size_t kMaskBytesPerBrick = 260;
inline size_t mask_alloc_bytes(long long nbricks) { return (size_t)nbricks * kMaskBytesPerBrick; }

// Per-frame pyramids of the largest and of the smallest accepted depth over
// square pixel tiles of 8, 16 and 32 pixels (float bits; where no pixel of the
// tile has an accepted depth, 0 in the largest and +inf in the smallest; the
// sign bit of a smallest-depth word is set when a pixel of the tile inside
// the image has no accepted depth):
// level L is a row-major grid of ceil(W / 2^(L+3)) x ceil(H / 2^(L+3)) tiles,
// the levels stored one after the other, the smallest-depth pyramid after the
// largest-depth one.
constexpr int kPyrLevels = 3;
struct PyrDims {
    int nx[kPyrLevels], ny[kPyrLevels];
    long long off[kPyrLevels + 1];  // off[kPyrLevels] = words of the whole pyramid
};
__host__ __device__ inline PyrDims pyr_dims(int width, int height)
{
    PyrDims d;
    long long acc = 0;
    for (int l = 0; l < kPyrLevels; ++l) {
        const int t = 8 << l;
        d.nx[l] = (width + t - 1) / t;
        d.ny[l] = (height + t - 1) / t;
        d.off[l] = acc;
        acc += (long long)d.nx[l] * d.ny[l];
    }
    d.off[kPyrLevels] = acc;
    return d;
}
// the same per level, without arrays (device code indexes levels at run time)
__host__ __device__ inline int pyr_tiles(int extent, int level) { return (extent + (8 << level) - 1) / (8 << level); }
__host__ __device__ inline long long pyr_level_off(int width, int height, int level)
{
    long long acc = 0;
    for (int l = 0; l < level; ++l) acc += (long long)pyr_tiles(width, l) * pyr_tiles(height, l);
    return acc;
}

// Work-list entry (table slot, packed brick coordinates bx | by << 10 | bz << 20):
// bit 30 marks a brick in front of every accepted depth of its pixels by
// more than mu, whose updated voxels all take f = 1 and no colour; bit 31 one
// whose voxels all project into the image onto accepted depths (with bit 30:
// every voxel inside the volume is updated with f = 1).
constexpr unsigned kListFree = 1u << 30;
constexpr unsigned kListFull = 1u << 31;
__host__ __device__ inline int packed_bz(unsigned packed) { return (int)((packed >> 20) & 1023u); }

struct Stats {
    unsigned long long swept, updated, band, bricks;
    unsigned long long rays, ray_samples, ray_skips, ray_hits;
    unsigned long long stream_up, stream_down;
};

// ---------------------------------------------------------------------------
// storage codecs: decode to / encode from float32 (F in units of mu, W count)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void decode_f16(uint32_t v, float &F, float &W)
{
    F = __half2float(__ushort_as_half((unsigned short)(v & 0xFFFFu)));
    W = (float)(v >> 16);
}
__device__ __forceinline__ uint32_t encode_f16(float F, float W)
{
    return (uint32_t)__half_as_ushort(__float2half_rn(F)) | ((uint32_t)W << 16);
}
__device__ __forceinline__ void decode_i16(uint32_t v, float &F, float &W)
{
    F = (float)(short)(v & 0xFFFFu) * (1.0f / 32767.0f);
    W = (float)(v >> 16);
}
__device__ __forceinline__ uint32_t encode_i16(float F, float W)
{
    int q = __float2int_rn(F * 32767.0f);
    q = max(-32767, min(32767, q));
    return (uint32_t)(unsigned short)(short)q | ((uint32_t)W << 16);
}

// decoded value of a just-encoded F (the sign that is actually stored)
__device__ __forceinline__ float stored_f16(float F)
{
    return __half2float(__float2half_rn(F));
}
__device__ __forceinline__ float stored_i16(float F)
{
    int q = __float2int_rn(F * 32767.0f);
    return (float)max(-32767, min(32767, q));
}

// ---------------------------------------------------------------------------
// host helper: kernel-node parameters for explicitly built CUDA graphs.  The
// argument values are held here until cudaGraphAddKernelNode or
// cudaGraphExecKernelNodeSetParams has copied them.
// ---------------------------------------------------------------------------
template <typename... Args>
struct NodeArgs {
    std::tuple<Args...> vals;
    void *ptrs[sizeof...(Args)];
    explicit NodeArgs(Args... a) : vals(a...) { fill(std::index_sequence_for<Args...>{}); }
    template <size_t... I>
    void fill(std::index_sequence<I...>) { ((ptrs[I] = (void *)&std::get<I>(vals)), ...); }
    cudaKernelNodeParams params(const void *func, dim3 grid, dim3 block)
    {
        cudaKernelNodeParams p{};
        p.func = const_cast<void *>(func);
        p.gridDim = grid;
        p.blockDim = block;
        p.sharedMemBytes = 0;
        p.kernelParams = ptrs;
        p.extra = nullptr;
        return p;
    }
};

// Add (exec == null) or update (exec != null) one kernel node.
inline cudaError_t graph_node(cudaGraph_t g, cudaGraphExec_t exec, cudaGraphNode_t *node,
                              cudaGraphNode_t dep, const cudaKernelNodeParams &p)
{
    if (exec) return cudaGraphExecKernelNodeSetParams(exec, *node, &p);
    return cudaGraphAddKernelNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, &p);
}

// Arguments of the raycast backward kernel (mv_backward.cu).
struct BackwardArgs {
    const VolDev *vols;
    int nvol;
    float *const *grad_tsdf;  // per table slot: dense float32 [z][y][x], or null
    const float *pose_f;      // per pose: R (9, row-major) and t (3) of the camera-to-world pose, float32
    const float *cam_f;       // per pose and table slot: camera position in the volume's voxel coordinates
                              // (t / s - h_t, computed in double, rounded once)
    int n_poses;
    float fx, fy, cx, cy;
    int width, height;
    const float *depth;       // n x h x w (forward tau*)
    const int *vol_id;        // n x h x w
    const float *grad_depth;  // n x h x w or null
    const float *grad_rgb;    // n x h x w x 3 or null
    float *grad_pose;         // n x 6 (written by the reduction)
    float *partial;           // n x (CTAs per pose) x 6 per-CTA sums of the pose gradient
    // L1 mode (ref_depth not null): grad_depth / grad_rgb are not read; each
    // pixel's are those of the L1 loss of the render against the reference
    const uint8_t *rgba;      // n x h x w x 4 (forward colour)
    const float *ref_depth;   // n x h x w
    const uint8_t *ref_rgba;  // n x h x w x 4
    float colour_weight;
    const unsigned *l1_count; // pixels valid in both renders (l1_stats_kernel)
};

// Scratch of the L1 statistics (32-bit words): [0] CTAs done, [1] pixels
// valid in both renders, then per CTA its colour sum (64-bit), its count and
// its depth sum (float).
constexpr int kL1Ctas = 592;
constexpr size_t kL1ScratchBytes = 4 * (2 + 4 * (size_t)kL1Ctas);

// element offset of voxel (x, y, z) in brick-major order
__device__ __forceinline__ long long vox_offset(const VolDev &v, int x, int y, int z)
{
    const long long b = ((long long)(z >> 3) * v.nb[1] + (y >> 3)) * v.nb[0] + (x >> 3);
    return b * kBrickVox + (((z & 7) << 6) | ((y & 7) << 3) | (x & 7));
}

}  // namespace mv
