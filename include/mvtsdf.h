/*
 * mvtsdf.h -- C ABI of the B300 multi-volume TSDF mapping library.
 *
 * The library implements the data-parallel hot path of the multi-volume
 * RGB-D mapper of Salvato, Finman and Leonard, "Multi-Volume High Resolution
 * RGB-D Mapping with Dynamic Volume Placement" (arXiv 1511.07106):
 *   - a set H of TSDF subvolumes h = (h_l, h_r, h_t) that can be added and
 *     removed at any frame (Sec. Dynamic Volume Allocation, Input and Output;
 *     Sec. Insertion and Removal);
 *   - projective TSDF + colour integration of a depth (+RGB) frame into every
 *     active volume (Sec. Volumetric Integration; Algorithm 1, first loop);
 *   - the per-pixel raycast of those volumes into depth / normal / colour /
 *     vertex maps, all volumes writing one map where the shortest ray distance
 *     wins (Sec. Raycasting; Algorithm 1, second loop);
 *   - moving a volume between GPU memory and host memory
 *     (Sec. Memory Passing; the upload and download steps of Algorithm 1).
 *
 * Conventions shared by every call:
 *   - Poses are 4x4 row-major camera-to-world matrices T = [R | t] in double
 *     precision (Sec. Depth Map Conversion, T^i = [R^i | t^i]).  Camera frame:
 *     x right, y down, z forward.
 *   - Voxel i of a volume with lattice offset h_t and pitch s sits at world
 *     position (h_t + i) * s (Sec. Volumetric Integration, t_s = t_l + h_t).
 *     Volumes whose offsets differ by integer multiples of (h_r - 2) tile space
 *     with the paper's two-voxel overlap (Sec. Initialization).
 *   - Depth is float32 z-depth in metres, row-major height x width; a value
 *     <= 0, NaN, or outside [z_min, z_max] is no measurement.  RGB is uint8
 *     height x width x 3, registered to depth with the same intrinsics.
 *   - TSDF values are stored in units of the truncation distance mu
 *     (range [-1, 1]); weights count frames, capped at w_max.
 *   - Device buffers passed in are owned by the caller and must stay valid
 *     until the work queued on `stream` has finished.  Volume storage in GPU
 *     memory and in pinned host memory is owned by the library.
 *   - Device buffers of floats, ints and 8-bit RGBA start on a 4-byte
 *     boundary, 64-bit keys and edge ids on an 8-byte one (RGB frames,
 *     3 bytes a pixel, may start anywhere); a call given another pointer
 *     returns MV_ERR_ARG and queues nothing.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous with respect to the
 *     host unless stated otherwise.
 *   - Every call returns an mv_status; no call aborts or throws.  The message
 *     of the last failure on a context is available from mv_last_error().
 *   - A context is not thread-safe: serialise calls on one context.
 */
#ifndef MVTSDF_H
#define MVTSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mv_ctx mv_ctx;

typedef enum {
    MV_OK = 0,
    MV_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad enum) */
    MV_ERR_OOM = 2,            /* GPU or pinned host allocation failed */
    MV_ERR_CUDA = 3,           /* a CUDA runtime call failed (message in mv_last_error) */
    MV_ERR_NOT_FOUND = 4,      /* no volume with that id */
    MV_ERR_NOT_RESIDENT = 5,   /* the volume is swapped out to host memory */
    MV_ERR_BUSY = 6,           /* operation conflicts with the volume's state */
    MV_ERR_DEVICE_TIMEOUT = 7, /* a bounded device-side loop gave up (status word set) */
    MV_ERR_CAPACITY = 8        /* more volumes / pixels than the library's fixed limits */
} mv_status;

/* TSDF storage format of one volume.  F32: float32 TSDF + float32 weight
 * (8 bytes per voxel).  F16: IEEE half TSDF (round to nearest even) + uint16
 * weight (4 bytes).  I16: int16 TSDF = round(F * 32767) clamped to +-32767 +
 * uint16 weight (4 bytes).  Every format adds 4 bytes of RGBA8 colour whose
 * alpha byte is the colour weight.  The update itself is computed in float32
 * for every format. */
typedef enum { MV_TSDF_F32 = 0, MV_TSDF_F16 = 1, MV_TSDF_I16 = 2 } mv_tsdf_fmt;

/* Pinhole intrinsics K (Sec. Input and Output): pixel (x, y) with integer
 * coordinates is the pixel centre; a camera point (X, Y, Z) projects to
 * u = fx X / Z + cx, v = fy Y / Z + cy. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
} mv_intrinsics;

/* Method parameters (the paper leaves all of them unstated). */
typedef struct {
    float trunc_voxels;  /* truncation distance mu, in voxels of each volume (default 4) */
    float w_max;         /* weight cap; <= 65535 for F16/I16 volumes (default 128) */
    int32_t color_w_max; /* colour weight cap, 1..255 (default 255) */
    float z_min, z_max;  /* accepted depth range and raycast range, metres (default 0, +inf) */
    float ray_step;      /* raycast sample spacing in voxels, [1/64, 1] (default 1) */
    int32_t n_bisect;    /* bisection steps inside the bracket before the final secant (default 8) */
} mv_config;

/* One subvolume h = (h_l, h_r, h_t) (Sec. Initialization): h_l = voxel_size * h_r. */
typedef struct {
    int32_t h_t[3];      /* lattice offset in voxels */
    int32_t h_r[3];      /* voxels per axis, each >= 2 */
    float voxel_size;    /* pitch s in metres, > 0 */
    int32_t fmt;         /* mv_tsdf_fmt */
} mv_volume_desc;

typedef struct {
    mv_volume_desc desc;
    int32_t resident;    /* 1: in GPU memory, 0: swapped out to pinned host memory */
    int32_t reserved;
    uint64_t device_bytes; /* GPU bytes held by the volume (voxels, colour, flags and the raycast's
                              derived bit masks of 256 bytes per 8^3 brick) */
    uint64_t host_bytes;   /* pinned host bytes held by the volume */
} mv_volume_info;

/* Work counters accumulated on the device since the last reset. */
typedef struct {
    uint64_t swept;       /* integration: voxels examined (voxels of bricks in the view frustum) */
    uint64_t updated;     /* integration: voxels whose TSDF and weight were updated */
    uint64_t band;        /* integration: voxels whose colour was updated (|sdf| < mu) */
    uint64_t bricks;      /* integration: 8x8x8 bricks processed */
    uint64_t rays;        /* raycast: pixels marched */
    uint64_t ray_samples; /* raycast: grid samples evaluated by trilinear interpolation */
    uint64_t ray_skips;   /* raycast: whole-brick shortcuts taken */
    uint64_t ray_hits;    /* raycast: pixels with a surface hit */
    uint64_t stream_up;   /* mv_frame_streamed: bricks uploaded to a staging slot */
    uint64_t stream_down; /* mv_frame_streamed: bricks written back to host copies */
} mv_stats;

/* Kernel kinds counted and timed by mv_get_timings. */
enum {
    MV_KERNEL_SETUP = 0,       /* per-call camera constants of every volume */
    MV_KERNEL_BRICK_LIST = 1,  /* frustum work list of bricks (batched calls: super bricks, then their bricks) */
    MV_KERNEL_INTEGRATE = 2,   /* TSDF + colour update of the listed bricks */
    MV_KERNEL_RAYCAST = 3,     /* per-pixel march, refinement, shading and merge */
    MV_KERNEL_FLAGS = 4,       /* brick summaries recomputed after a host write */
    MV_KERNEL_CELL_FLAGS = 5,  /* raycast cell masks and step-over flags refreshed after an integration */
    MV_KERNEL_BACKWARD = 6,    /* raycast gradients */
    MV_KERNEL_FRAME_GRAPH = 7, /* one mv_frame graph (its 6 or 7 kernels are also counted by kind) */
    MV_KERNEL_DEPTH_MAX = 8,   /* the frame's depth-tile pyramids and farthest accepted depth (brick list bounds) */
    MV_KERNEL_EXTRACT = 9,     /* surface points of a volume */
    MV_KERNEL_DEPTH_MAPS = 10, /* vertex / normal maps of a depth frame */
    MV_KERNEL_ICP = 11,        /* one point-to-plane ICP linearisation */
    MV_KERNEL_STREAM = 12,     /* brick gather / scatter of mv_frame_streamed */
    MV_KERNEL_KINDS = 13
};

typedef struct {
    uint64_t launches[MV_KERNEL_KINDS]; /* kernels launched, by kind */
    double ms[MV_KERNEL_KINDS];         /* summed device time, by kind, while timing is on */
    uint64_t timed[MV_KERNEL_KINDS];    /* launches included in ms */
} mv_timings;

/* Library version string (static storage). */
const char *mv_version(void);

/* Fill *out with the default configuration.  MV_ERR_ARG if out is NULL. */
mv_status mv_config_default(mv_config *out);

/* Create a context on CUDA device `device` (made current on the calling
 * thread).  cfg may be NULL for defaults.  Fails with MV_ERR_ARG on invalid
 * parameters, MV_ERR_CUDA if the device cannot be used. */
mv_status mv_create(const mv_config *cfg, int32_t device, mv_ctx **out);

/* Wait for all of the context's work, free every volume (GPU and host) and
 * the context.  NULL is accepted. */
mv_status mv_destroy(mv_ctx *ctx);

/* Message of the last failed call on ctx (static or context-owned storage,
 * valid until the next call on ctx). */
const char *mv_last_error(const mv_ctx *ctx);

/* Add a volume (Sec. Dynamic Volume Allocation: "a volume can be added to the
 * set at any point").  Allocates its storage in GPU memory and clears it to
 * F = 0, W = 0 (unobserved), colour 0, ordered on the context's internal
 * stream before any later call.  *out_id receives an id that is never
 * reused.  MV_ERR_OOM if GPU memory is exhausted (nothing is allocated),
 * MV_ERR_CAPACITY beyond 4096 volumes. */
mv_status mv_add_volume(mv_ctx *ctx, const mv_volume_desc *desc, int32_t *out_id);

/* Remove a volume from the set and free its GPU and host storage once work
 * already queued on it has finished (Sec. Insertion and Removal). */
mv_status mv_remove_volume(mv_ctx *ctx, int32_t id);

/* Describe a volume.  MV_ERR_NOT_FOUND for an unknown id. */
mv_status mv_query(mv_ctx *ctx, int32_t id, mv_volume_info *out);

/* List volume ids in ascending order: writes min(count, cap) ids to ids
 * (may be NULL when cap == 0) and the total into *count. */
mv_status mv_list_volumes(mv_ctx *ctx, int32_t *ids, int32_t cap, int32_t *count);

/* Integrate one frame into every resident volume in one batched pass: a
 * work list of the 8x8x8 bricks that intersect the view frustum of every
 * resident volume is built on the device, then one persistent kernel updates
 * them (Sec. Volumetric Integration).  depth: device float32 [height*width];
 * rgb: device uint8 [height*width*3] or NULL (no colour update).  Volumes
 * that are swapped out are skipped, as the paper processes only active
 * volumes.  Asynchronous on `stream`. */
mv_status mv_integrate(mv_ctx *ctx, const float *depth, const uint8_t *rgb,
                       const mv_intrinsics *K, const double T_c2w[16], void *stream);

/* The same update for one volume only (the paper's per-volume step of
 * Algorithm 1).  MV_ERR_NOT_RESIDENT if the volume is swapped out. */
mv_status mv_integrate_volume(mv_ctx *ctx, int32_t id, const float *depth, const uint8_t *rgb,
                              const mv_intrinsics *K, const double T_c2w[16], void *stream);

/* Raycast every resident volume into one set of maps in one pass; for each
 * pixel the hit with the smallest ray distance wins, exact ties going to the
 * lower volume id (Sec. Raycasting).  Output device buffers (each may be
 * NULL): depth float32 [h*w] (z-depth, 0 = no hit), normal float32 [h*w*3]
 * (unit, world frame, facing the camera; 0 where the hit cell has an
 * unobserved corner), rgba uint8 [h*w*4] (A = 255 on hits, 0 otherwise),
 * vertex float32 [h*w*3] (world frame), vol_id int32 [h*w] (-1 = no hit).
 * Asynchronous on `stream`. */
mv_status mv_raycast(mv_ctx *ctx, const mv_intrinsics *K, const double T_c2w[16],
                     float *depth, float *normal, uint8_t *rgba, float *vertex, int32_t *vol_id,
                     void *stream);

/* The raycast of mv_raycast for n_views views of the same resident volumes
 * in one kernel launch (the views of a batch of camera poses, e.g. for pose
 * refinement).  T_c2w: host, n_views x 16 doubles (1 <= n_views <= 65535).
 * Each output (device, may be NULL) holds n_views maps one after the other,
 * in the layout of mv_raycast: depth and vol_id n x h x w, normal and vertex
 * n x h x w x 3, rgba n x h x w x 4.  View k's maps equal those of
 * mv_raycast at pose k, bit for bit.  Asynchronous on `stream`. */
mv_status mv_raycast_batch(mv_ctx *ctx, const mv_intrinsics *K, const double *T_c2w, int32_t n_views,
                           float *depth, float *normal, uint8_t *rgba, float *vertex, int32_t *vol_id,
                           void *stream);

/* One frame of the paper's per-frame loop: integrate the frame into every
 * resident volume, then raycast every resident volume at the same pose, as
 * one CUDA graph launch (6 kernels; 7 with the two-level work list).  Same semantics and outputs as
 * mv_integrate followed by mv_raycast.  The graph is built on the first call
 * and rebuilt when the set of resident volumes or the image size changes;
 * otherwise each call only updates the graph's kernel parameters (pose and
 * buffers).  While timing is on, the graph is timed as a whole
 * (MV_KERNEL_FRAME_GRAPH). */
mv_status mv_frame(mv_ctx *ctx, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                   const double T_c2w[16], float *depth_out, float *normal, uint8_t *rgba,
                   float *vertex, int32_t *vol_id, void *stream);

/* One frame of the paper's per-frame loop from and to host memory
 * (Algorithm 1: upload the frame, integrate it into every resident volume,
 * raycast them, download the maps).  depth (float32 h*w) and rgb (uint8
 * h*w*3, or NULL for no colour update) are HOST buffers; depth_out (float32
 * h*w), normal (float32 h*w*3), rgba (uint8 h*w*4), vertex (float32 h*w*3)
 * and vol_id (int32 h*w) are HOST output buffers, each may be NULL (that map
 * is not downloaded).  The maps are those of mv_frame.  Page-locked host
 * buffers make the copies asynchronous; pageable ones also work, the driver
 * then stages them.  The call only enqueues work and returns a ticket: the
 * library keeps two device buffer sets (frame in, maps out) and three
 * internal streams, one per stage (upload, kernels, download), so the upload
 * of the next frame and the download of the previous one overlap the kernels
 * of this one.  mv_frame_host_wait(ctx, ticket) blocks until that frame's
 * maps are in its output buffers; until then every buffer of the frame must
 * stay valid and unmodified.  Calls on one context still execute in call
 * order.  The buffers are allocated on the first call and again when the
 * image size changes (which first waits for the frames in flight). */
mv_status mv_frame_host(mv_ctx *ctx, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                        const double T_c2w[16], float *depth_out, float *normal, uint8_t *rgba,
                        float *vertex, int32_t *vol_id, uint64_t *ticket);

/* Wait until the frame of `ticket` (from mv_frame_host) has been downloaded
 * (and its input buffers are no longer read).  MV_ERR_ARG for a ticket not
 * yet issued. */
mv_status mv_frame_host_wait(mv_ctx *ctx, uint64_t ticket);

/* Full-cover out-of-core frame (Sec. Volumetric Integration and
 * Sec. Raycasting, Algorithm 1: every volume is uploaded, integrated,
 * raycast and downloaded again in every frame).  Resident volumes are
 * integrated and raycast in place, as by mv_frame; then every swapped-out
 * volume passes through one of n_slots (1..4) device staging slots: on one
 * side stream its flags and the bricks the frame can read (those whose cells
 * meet the view frustum, found from the pose) are uploaded, the bricks by a
 * kernel that reads the pinned host copy directly; it is integrated and raycast
 * into the same maps on `stream` (nearest hit wins, ties to the lower id, so
 * the maps equal those of all volumes resident); on a second side stream its
 * flags and the bricks the integration changed are written back to the host
 * copy.  The uploads and write-backs of one slot overlap the kernels of
 * another.  mv_get_stats counts the bricks moved (stream_up, stream_down).  The volumes stay swapped out.  The slots (sized for the largest
 * swapped-out volume) are kept by the context for later calls.  `stream`
 * waits for the last download; later swap-in, read and write calls wait for
 * the downloads of their volume.  depth_out and vol_id are required.
 * MV_ERR_ARG for n_slots outside 1..4; MV_ERR_OOM when the slots do not fit. */
mv_status mv_frame_streamed(mv_ctx *ctx, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                            const double T_c2w[16], float *depth_out, float *normal, uint8_t *rgba,
                            float *vertex, int32_t *vol_id, int32_t n_slots, void *stream);

/* Raycast one volume and merge its hits into the maps (the paper's
 * per-volume raycast, in which every volume writes into one shared map).  With
 * first != 0 the maps are (re)initialised by this call; otherwise a pixel is
 * overwritten only when this volume's hit is nearer, or equally near with a
 * lower id.  depth and vol_id are required (they carry the merge state);
 * the other outputs may be NULL. */
mv_status mv_raycast_volume(mv_ctx *ctx, int32_t id, int32_t first, const mv_intrinsics *K,
                            const double T_c2w[16], float *depth, float *normal, uint8_t *rgba,
                            float *vertex, int32_t *vol_id, void *stream);

/* Launch shapes chosen by mv_autotune (or set by mv_set_tuning). */
typedef struct {
    int32_t raycast_tile;          /* 0: 16x8 CTA of 8x4 warps, 1: 32x4 of 8x4, 2: 8x16 of 8x4,
                                      3: 32x4 CTA of 32x1 warps */
    int32_t integrate_ctas_per_sm; /* persistent integration grid = SMs x this */
    float raycast_ms[4];           /* median per tile shape (mv_autotune only) */
    float integrate_ms[5];         /* median for 2, 4, 6, 8, 10 CTAs per SM (mv_autotune only;
                                      0 where not measured) */
    int32_t work_list_levels;      /* work list of the batched calls: 1 one thread per brick,
                                      2 super bricks in view first, then their bricks; 0 automatic
                                      (2 from 2^20 resident bricks on).  Same list either way. */
} mv_tuning;

/* Choose the raycast pixel tile and the integration grid size by timing the
 * candidates on this frame and view (median of 5 launches each; the current
 * choice is kept unless another candidate is more than 3 % faster): the
 * raycast runs on the resident volumes (it changes no state), the integration
 * on temporary scratch storage shaped like the largest volume in view (the
 * map is not modified; with no volume in view the grid is kept).  Synchronous;
 * the choice applies to every later call of the context (results do not
 * depend on it, only speed). */
mv_status mv_autotune(mv_ctx *ctx, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                      const double T_c2w[16], mv_tuning *out, void *stream);

/* Set / read the launch shapes (raycast_tile, integrate_ctas_per_sm,
 * work_list_levels); mv_autotune keeps work_list_levels. */
mv_status mv_set_tuning(mv_ctx *ctx, const mv_tuning *t);
mv_status mv_get_tuning(mv_ctx *ctx, mv_tuning *t);

/* Gradient target of mv_raycast_backward: the TSDF gradient of volume `id`
 * is accumulated (+=) into grad_tsdf, a device float32 array in the linear
 * order of mv_read_volume (h_r[0] * h_r[1] * h_r[2] values). */
typedef struct {
    int32_t id;
    float *grad_tsdf;
} mv_grad_target;

/* Gradients of raycast depth and colour (not in the paper; the
 * differentiable raycast used for pose refinement).  For n_poses views that
 * were raycast with mv_raycast (depth and vol_id of each view, device,
 * n_poses x height x width, unchanged since), and upstream gradients
 * grad_depth (dL/d depth, n x h x w) and grad_rgb (dL/d colour with colour in
 * [0, 1], n x h x w x 3), either may be NULL:
 *   grad_pose (device, n x 6, overwritten) receives dL/dxi for the left
 *   perturbation T(xi) = exp(xi^) T of each pose, xi = (rho, phi) in the
 *   world frame (rho translation in metres, phi rotation in radians);
 *   each target's grad_tsdf receives += dL/dF for that volume's TSDF values
 *   (F in units of the truncation distance).
 * The hit cell is re-derived from depth and vol_id (no per-step storage).
 * Colour is differentiated as the unrounded trilinear colour of the hit cell
 * (the forward's 8-bit rounding is passed straight through).  Pixels with no
 * hit, an unobserved corner, grazing incidence or a hit within 1e-3 voxel of
 * a cell face contribute nothing.  T_c2w: host, n_poses x 16 doubles.
 * Asynchronous on `stream`.  grad_pose is summed in a fixed order (the same
 * bits on every run); the TSDF gradients are summed by float atomics, whose
 * order, and so the last bits of the result, vary between runs. */
mv_status mv_raycast_backward(mv_ctx *ctx, const mv_intrinsics *K, const double *T_c2w,
                              int32_t n_poses, const float *depth, const int32_t *vol_id,
                              const float *grad_depth, const float *grad_rgb, float *grad_pose,
                              const mv_grad_target *targets, int32_t n_targets, void *stream);

/* The L1 loss of pose refinement and its pose gradient in one call (not in
 * the paper; the loss the Python binding's refinement minimises).  For
 * n_poses views raycast with mv_raycast_batch (depth, rgba and vol_id,
 * device, n x h x w, and n x h x w x 4 bytes for rgba) against reference
 * renders ref_depth (n x h x w) and ref_rgba (n x h x w x 4 bytes, A unused):
 * with the pixels valid in both renders (depth > 0 in each) counted as
 * n_valid, the loss is the mean over them of |depth - ref_depth| +
 * colour_weight * sum over R, G, B of |c - ref_c|, colours c = byte / 255;
 * its gradient at a pixel is w sign(depth - ref_depth) for depth and
 * (colour_weight sign(c - ref_c)) w for colour, w = 1 / n_valid (1 / 1 when
 * none is valid, so every gradient is then 0), 0 elsewhere.  grad_pose
 * (device, n x 6, overwritten) receives that gradient carried through the
 * raycast as mv_raycast_backward carries grad_depth and grad_rgb (the same
 * per-pixel values in the same order: the same bits); loss (device, one
 * float) receives the loss, its sums in a fixed order.  One kernel adds the
 * statistics, then the backward kernel forms each pixel's gradient itself:
 * no per-pixel gradient buffers.  Every buffer 4-byte aligned (else
 * MV_ERR_ARG, nothing launched).  Asynchronous on `stream`; calls of one
 * context share its statistics scratch, so calls on different streams must
 * not overlap. */
mv_status mv_raycast_backward_l1(mv_ctx *ctx, const mv_intrinsics *K, const double *T_c2w,
                                 int32_t n_poses, const float *depth, const uint8_t *rgba,
                                 const int32_t *vol_id, const float *ref_depth, const uint8_t *ref_rgba,
                                 float colour_weight, float *grad_pose, float *loss, void *stream);

/* Move a volume to pinned host memory (the paper's download to the CPU, Algorithm 1)
 * on the library's swap stream, after the work already queued on `stream`;
 * its GPU memory is released once the copy has finished.  From this call on
 * the volume is skipped by mv_integrate / mv_raycast.  MV_ERR_OOM if pinned
 * memory cannot be allocated (the volume then stays resident). */
mv_status mv_swap_out(mv_ctx *ctx, int32_t id, void *stream);

/* Bring a swapped-out volume back to GPU memory (the paper's upload to the GPU, Algorithm 1) on the swap
 * stream; later calls on any stream wait for the copy.  MV_ERR_OOM if GPU
 * memory is exhausted (the volume stays on the host). */
mv_status mv_swap_in(mv_ctx *ctx, int32_t id, void *stream);

/* Synchronous copy of a volume's state to host memory in linear order
 * (index ((z * h_r[1]) + y) * h_r[0] + x).  host_fw receives the raw storage
 * per voxel: F32 -> 2 x float32 (F, W); F16 -> uint32 (bits 0-15 IEEE half F,
 * bits 16-31 uint16 W); I16 -> uint32 (bits 0-15 int16 F, bits 16-31 uint16 W).
 * host_rgba receives 4 bytes per voxel (may be NULL).  Works for resident
 * and swapped-out volumes. */
mv_status mv_read_volume(mv_ctx *ctx, int32_t id, void *host_fw, uint8_t *host_rgba);

/* Synchronous copy of a box of a volume's voxels to host memory: voxels
 * lo[a] .. lo[a] + n[a] - 1 along each axis a = x, y, z (0 <= lo[a],
 * n[a] >= 1, lo[a] + n[a] <= h_r[a]), in the layout of mv_read_volume over the
 * box (index ((z * n[1]) + y) * n[0] + x).  host_rgba may be NULL.  A
 * resident volume's box is gathered on the GPU, a swapped-out one's from its
 * host copy.  For reading the observed part of a large volume without
 * copying all of it.  MV_ERR_ARG for a box outside the volume. */
mv_status mv_read_box(mv_ctx *ctx, int32_t id, const int32_t lo[3], const int32_t n[3], void *host_fw,
                      uint8_t *host_rgba);

/* Synchronous overwrite of a volume's state from host memory in the layout of
 * mv_read_volume (host_rgba NULL keeps the colour).  Used to prefill volumes
 * and to restore checkpoints. */
mv_status mv_write_volume(mv_ctx *ctx, int32_t id, const void *host_fw, const uint8_t *host_rgba);

/* Synchronous copy of a volume's per-brick summary flags (one byte per
 * 8x8x8 brick, brick index (bz * nby + by) * nbx + bx with nb = ceil(h_r / 8);
 * bit 0: every voxel of the brick observed with F > 0, bit 1: no voxel of the
 * brick observed, bit 2: no voxel of the brick observed with F <= 0).  The raycast relies on these summaries to step over whole
 * bricks; they are exposed so that their soundness can be checked.
 * MV_ERR_ARG if cap is smaller than the brick count. */
mv_status mv_read_brick_flags(mv_ctx *ctx, int32_t id, uint8_t *host_flags, uint64_t cap);

/* Read (and optionally reset) the integration counters; synchronises the
 * context's work. */
mv_status mv_get_stats(mv_ctx *ctx, mv_stats *out, int32_t reset);

/* Turn per-kernel timing on or off.  While on, every kernel launch is
 * bracketed by two CUDA events recorded on the launching stream. */
mv_status mv_set_timing(mv_ctx *ctx, int32_t enable);

/* Launch counts and (while timing was on) summed device time per kernel kind
 * since the last reset; synchronises the context's work. */
mv_status mv_get_timings(mv_ctx *ctx, mv_timings *out, int32_t reset);

/* ---------------------------------------------------------------------------
 * Integration without allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate GPU memory themselves or through the library -- code that
 * runs inside a host framework's memory budget, inside a pre-sized memory
 * pool, or where a cudaMalloc would synchronise the device at a bad time.
 * It integrates one frame into one volume whose storage the caller owns and
 * passes in, and it allocates nothing: no context, no cudaMalloc, no
 * cudaFree.  Its working memory (the frustum brick list and per-call
 * constants) is one fixed array of about 2 MiB compiled into the library,
 * which every GPU that loads the library keeps until the process exits.
 *
 * The caller's storage uses the library's brick layout: the volume is padded
 * to nb = ceil(h_r / 8) bricks per axis; brick (bx, by, bz) is stored at
 * brick index (bz * nby + by) * nbx + bx, 512 voxels each, voxel (lx, ly, lz)
 * at (lz * 8 + ly) * 8 + lx inside its brick.  fw holds 8 bytes per voxel for
 * MV_TSDF_F32 (float32 F, float32 W) and 4 bytes for MV_TSDF_F16 / I16 (the
 * codes of mv_read_volume); rgba 4 bytes per voxel; brick_flags 1 byte per
 * brick (the summaries of mv_read_brick_flags).  A new volume starts with fw
 * and rgba all zero and every brick flag equal to 6 (nothing observed, hence
 * nothing observed at or behind a surface).  fw must be 16-byte aligned.
 * ------------------------------------------------------------------------- */

/* Largest volume mv_integrate_noalloc accepts, in 8x8x8 bricks (64^3 bricks:
 * a 512^3 volume). */
#define MV_NOALLOC_MAX_BRICKS 262144

typedef struct {
    mv_volume_desc desc;  /* h_t, h_r, voxel_size, fmt */
    void *fw;             /* device, brick-major TSDF + weight */
    uint8_t *rgba;        /* device, brick-major RGBA8 */
    uint8_t *brick_flags; /* device, one byte per brick */
} mv_volume_view;

/* Integrate one frame into a caller-owned volume, allocating nothing.  cfg
 * may be NULL for defaults; the configurations it accepts are those
 * mv_create accepts.  Works on the current CUDA device.  Each call whose
 * stream is not being captured looks up the device address of the library's
 * fixed working array in the current context (a device reset moves it); a
 * call on a capturing stream reuses the address found by the device's last
 * uncaptured call, so make one call on each device before any stream capture
 * (and again after a device reset).  All calls share that one array: calls
 * whose work overlaps on the GPU (on different streams, or from different
 * threads) race and must be serialised by the caller.  Returns
 * MV_ERR_CAPACITY, without launching anything, for a volume of more than
 * MV_NOALLOC_MAX_BRICKS bricks; MV_ERR_ARG for a null or misaligned pointer
 * or an invalid size, format, configuration or frame; MV_ERR_CUDA for a first
 * call on a device made during a stream capture.  Asynchronous on `stream`
 * otherwise. */
mv_status mv_integrate_noalloc(const mv_volume_view *vol, const mv_config *cfg, const float *depth,
                               const uint8_t *rgb, const mv_intrinsics *K, const double T_c2w[16],
                               void *stream);

/* Surface points of one resident volume: the point cloud that stands for a
 * volume once it leaves the map (Sec. Insertion and Removal); their number is
 * the paper's resolution measure (Table 1, vertices).  One point per edge
 * between 6-neighbour voxels i and i + e_a (a = x, y, z; both inside the
 * volume) that are both observed (W > 0) and on different sides of the
 * surface, (F_i > 0) != (F_{i+e_a} > 0): the zero of the linear
 * interpolation, p = (h_t + i + t e_a) * voxel_size, t = F_i / (F_i - F_{i+e_a}).
 * Its colour is the linear interpolation of the two voxels' RGB at t, rounded
 * half up; its edge id is 3 * (z * h_r[1] + y) * h_r[0] + 3 * x + a for
 * i = (x, y, z).  Outputs are device arrays for cap points, each may be
 * NULL: xyz float32 [3 cap], rgb uint8 [3 cap], edge uint64 [cap].  Points come
 * in no particular order; volumes that share voxel planes each report the
 * points of their own edges.  *n receives the number of points (min(n, cap)
 * written).  Blocks until done.  MV_ERR_CAPACITY when n > cap;
 * MV_ERR_NOT_RESIDENT for a swapped-out volume. */
mv_status mv_extract_points(mv_ctx *ctx, int32_t id, float *xyz, uint8_t *rgb, uint64_t *edge, uint64_t cap,
                            uint64_t *n, void *stream);

/* ---------------------------------------------------------------------------
 * Depth-map conversion and camera tracking (Sec. Depth Map Conversion;
 * Sec. Camera Tracking, point-to-plane ICP with projective data association
 * as in KinectFusion).
 * ------------------------------------------------------------------------- */

/* Vertex and normal maps of a depth frame: v = K^-1 [x, y, 1]^T D(x, y) for
 * every pixel with a valid depth (> 0, inside the context's [z_min, z_max]),
 * and n = (v(x+1, y) - v(x, y)) x (v(x, y+1) - v(x, y)), normalised and turned
 * to face the camera, where the three depths are valid (not in the last
 * column or row).  With T_c2w both are moved to the world frame (v -> R v + t,
 * n -> R n); with T_c2w NULL they stay in the camera frame.  Invalid vertices
 * and normals are 0.  vertex and normal are device float32 [height*width*3].
 * Asynchronous on `stream`. */
mv_status mv_depth_to_maps(mv_ctx *ctx, const float *depth, const mv_intrinsics *K, const double T_c2w[16],
                           float *vertex, float *normal, void *stream);

typedef struct {
    int32_t iterations; /* Gauss-Newton steps of mv_track, 0..1000 */
    float dist;         /* association distance threshold, metres, > 0 */
    float cos_min;      /* association normal threshold: cos of the largest angle, -1..1 */
} mv_icp_config;

typedef struct {
    double A[36];    /* sum of J^T J, row-major */
    double b[6];     /* sum of J^T r */
    double error;    /* sum of r^2 */
    int64_t inliers; /* associated pixels */
} mv_icp_system;

/* One point-to-plane linearisation.  vertex / normal: the current frame's
 * maps in its camera frame (mv_depth_to_maps with T NULL); model_vertex /
 * model_normal: world-frame maps of the same size seen from T_model (e.g.
 * the raycast of the previous frame; a normal of 0 marks a miss).  Each pixel
 * with a normal is moved by T_est (v_g = R v + t, n_g = R n), projected into
 * the model camera, and associated with the model vertex V and normal N at
 * the nearest pixel (floor(u + 1/2)) when |v_g - V| <= dist and
 * n_g . N >= cos_min.  With r = N . (V - v_g) and J = [N, v_g x N] (the twist
 * x = (rho, phi) moves v_g to v_g + rho + phi x v_g, so r changes by -J x)
 * it adds J^T J, J^T r, r^2 and 1.  Per-pixel terms, the sums of a thread,
 * within a warp and over a CTA's warps (pairwise trees) in FP32; the CTAs'
 * sums in FP64 on the host; every order fixed.  Blocks until the system is
 * on the host. */
mv_status mv_icp_linearize(mv_ctx *ctx, const float *vertex, const float *normal, const mv_intrinsics *K,
                           const double T_est[16], const float *model_vertex, const float *model_normal,
                           const double T_model[16], const mv_icp_config *cfg, mv_icp_system *out,
                           void *stream);

/* Track one frame: the depth frame's camera-frame maps, then cfg->iterations
 * Gauss-Newton steps from T_init: solve A x = b (Cholesky, FP64) and set
 * T <- exp(x^) T.  Stops early when fewer than 6 pixels associate or the
 * system is not positive definite.  The loop runs on the device: each step is
 * one kernel whose last CTA adds the partial sums in a fixed order
 * (compensated FP32 summation, about 48 bits), solves in FP64 and updates
 * the estimate in device memory, so the steps follow each other
 * without a host round trip.  T_out receives the estimate; last (may be
 * NULL) the system of the last linearisation.  Blocks until done (one
 * read-back at the end). */
mv_status mv_track(mv_ctx *ctx, const float *depth, const mv_intrinsics *K, const float *model_vertex,
                   const float *model_normal, const double T_model[16], const double T_init[16],
                   const mv_icp_config *cfg, double T_out[16], mv_icp_system *last, void *stream);

/* Hold `count` (0..4096) spare sets of pinned host buffers for volumes
 * shaped like `desc` (h_r and fmt), pinning the missing ones now (this call
 * takes as long as pinning them), so that a later first mv_swap_out of such a
 * volume need not wait while gigabytes of host memory are pinned.  Swap-outs
 * take spares first; buffers of removed volumes return to the spares while
 * fewer than `count` are held; 0 frees the spares.  MV_ERR_OOM when the host
 * cannot pin that much (the sets pinned so far are kept). */
mv_status mv_reserve_host(mv_ctx *ctx, const mv_volume_desc *desc, int32_t count);

/* The configuration the context was created with. */
mv_status mv_get_config(const mv_ctx *ctx, mv_config *out);

/* The CUDA device of the context (-1 for NULL). */
int32_t mv_get_device(const mv_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Dynamic volume placement (Sec. Dynamic Mapping for SLAM; Sec. Insertion and
 * Removal).  Space is cut into a lattice of cubic cells of cell_voxels voxels
 * (the paper's d_v - 2); the volume of cell k = (kx, ky, kz) has lattice
 * offset h_t = k * cell_voxels and volume_voxels voxels per axis (d_v), so
 * that the volumes of neighbouring cells share two voxel planes.  Each frame
 * the endpoint e = T (D K^-1 [x, y, 1]^T) of every pixel whose depth D is
 * valid (> 0, inside the context's [z_min, z_max]) is binned into its cell
 * l = floor(e / (cell_voxels * voxel_size)), in double precision with a fixed
 * operation order: xn = (x - cx) / fx, yn = (y - cy) / fy, p = (D xn, D yn, D),
 * e_a = ((R_a0 p_0 + R_a1 p_1) + R_a2 p_2) + t_a.  c(l) is the number of
 * endpoints in cell l.
 *
 * Policy of one update (after the frame's raycast, as the paper orders it):
 * cells that are not resident and have at least min_count endpoints are taken
 * by decreasing count (ties by increasing z, then y, then x).  While fewer
 * than max_volumes placed volumes are resident, each enters.  Then each
 * remaining one enters only by displacing the resident cell of lowest count
 * (ties: increasing z, y, x), and only when its count is larger than that
 * count times `hysteresis`; the first that is not stops the step.  A cell
 * enters by creating its volume (mv_add_volume) or, if it had one before, by
 * mv_swap_in; a displaced cell leaves by mv_swap_out (its volume keeps its
 * data in pinned host memory).  Placed volumes are ordinary volumes of the
 * context: every integrate / raycast / frame call sees the resident ones.
 * The placer does not own them; destroying it leaves them in the context.
 * ------------------------------------------------------------------------- */
typedef struct mv_placer mv_placer;

typedef struct {
    int32_t cell_voxels;   /* lattice spacing in voxels, >= 1 */
    int32_t volume_voxels; /* voxels per axis of a placed volume, cell_voxels..8192 */
    float voxel_size;      /* metres, > 0 */
    int32_t fmt;           /* mv_tsdf_fmt of placed volumes */
    int32_t max_volumes;   /* resident placed volumes at most, >= 1 */
    float hysteresis;      /* displacement factor, >= 1 */
    int32_t min_count;     /* fewest endpoints for a cell to be placed, >= 1 */
} mv_placement_config;

typedef struct {
    int32_t cells;    /* distinct cells with endpoints in this frame */
    int32_t added;    /* volumes created */
    int32_t restored; /* volumes swapped back in */
    int32_t evicted;  /* volumes swapped out */
    int32_t resident; /* placed volumes resident after the step */
} mv_placement_result;

/* MV_ERR_ARG for a NULL argument or a configuration outside the ranges above. */
mv_status mv_placer_create(mv_ctx *ctx, const mv_placement_config *cfg, mv_placer **out);
mv_status mv_placer_destroy(mv_placer *placer);
const char *mv_placer_last_error(const mv_placer *placer);

/* c(l) of one frame: writes min(n, cap) cells (3 int32 each, x y z) and
 * counts, sorted by increasing z, then y, then x, and the number of distinct
 * cells into *n.  depth is a device float32 [height*width] array.  Blocks
 * until the result is on the host.  MV_ERR_CAPACITY when n > cap (the first
 * cap are written) or when a cell coordinate is beyond +-2^20. */
mv_status mv_placer_histogram(mv_placer *placer, const float *depth, const mv_intrinsics *K,
                              const double T_c2w[16], int32_t *cells, uint32_t *counts, int32_t cap,
                              int32_t *n, void *stream);

/* One insertion / removal step on this frame's depth (policy above).  The
 * swaps are asynchronous (side stream, ordered after `stream`); out may be
 * NULL.  Errors of the add / swap calls are passed on. */
mv_status mv_placer_update(mv_placer *placer, const float *depth, const mv_intrinsics *K,
                           const double T_c2w[16], mv_placement_result *out, void *stream);

/* Placed volumes by increasing id: ids, their cells (3 int32 each) and
 * residency (1 or 0); min(n, cap) entries written, the total into *n. */
mv_status mv_placer_list(mv_placer *placer, int32_t *ids, int32_t *cells, int32_t *resident, int32_t cap,
                         int32_t *n);

/* Wait until all work of the context (all streams it used) has finished. */
mv_status mv_synchronize(mv_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Merge of maps raycast on different GPUs (volumes partitioned across GPUs).
 *
 * The paper merges the hits of all volumes per pixel by the shortest ray
 * distance (Sec. Raycasting, last paragraph), and the integration of
 * different volumes is independent (Sec. Comparison to KinectFusion), so the
 * volumes of one map can live on several GPUs: each raycasts its own
 * volumes (mv_raycast / mv_frame), packs its per-pixel hits into 64-bit keys
 * (mv_pack_hits), the keys are combined by an all-reduce MIN (e.g. NCCL),
 * each GPU clears the pixels it did not win and takes depth and volume id
 * from the winning key (mv_merge_hits), and an all-reduce SUM of normal,
 * colour and vertex maps completes every GPU's copy.  The merged maps equal
 * those of one GPU holding every volume, bit for bit.  Neither call needs a
 * context; both run on the current device, asynchronously on `stream`.
 * ------------------------------------------------------------------------- */

/* keys[p] = (bits of depth[p] << 32) | global id, where the global id of a
 * local volume id v is id_map[v] (id_map_len entries; id_map NULL with
 * id_map_len 0: the local id itself); INT64_MAX (no hit) where vol_id[p] < 0,
 * depth is not a positive finite value, or the id has no global id.  A hit
 * key is a non-negative int64 below INT64_MAX, so signed 64-bit MIN picks the
 * nearest hit, equal distances going to the lower global id (the single-GPU
 * tie rule).  depth: float32 [n] (ray distance tau = z-depth), vol_id: int32
 * [n], id_map: int32, keys: int64 [n], all device. */
mv_status mv_pack_hits(const float *depth, const int32_t *vol_id, const int32_t *id_map, int32_t id_map_len,
                       int64_t n, int64_t *keys, void *stream);

/* With best_keys the element-wise minimum of every GPU's keys and own_keys
 * this GPU's: depth[p] and vol_id[p] are set from best_keys (0 and -1 where
 * no GPU hit); normal[3 p..], rgba[p] (4 bytes, 4-byte aligned) and
 * vertex[3 p..] are cleared where this GPU's key is not the winner.  Each
 * output may be NULL.  All device arrays of n pixels. */
mv_status mv_merge_hits(const int64_t *best_keys, const int64_t *own_keys, int64_t n, float *depth,
                        int32_t *vol_id, float *normal, uint8_t *rgba, float *vertex, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MVTSDF_H */
