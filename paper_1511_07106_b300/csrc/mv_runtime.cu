// mv_runtime.cu -- host runtime behind the C ABI of include/mvtsdf.h.
//
// Owns the volume registry (the paper's set H of subvolumes, Sec. Dynamic
// Volume Allocation), the device table of resident volumes that the batched
// kernels index, the per-call scratch (brick work list, per-volume camera
// constants, counters), and the swap engine that moves volumes between GPU
// memory and pinned host memory on a side stream (Sec. Memory Passing).
//
// Ordering: every call that queues GPU work waits (cudaStreamWaitEvent) for
// the previous call's work, so calls on one context execute in call order
// whatever streams they are given.  Volume storage is allocated and freed
// stream-ordered (cudaMallocAsync / cudaFreeAsync) on the swap stream, so
// swapping a volume out never blocks the host or the compute stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "mv_internal.cuh"
#include "mv_pinned.h"

namespace mv {
constexpr int kMaxStreamSlots = 4;
cudaError_t launch_frame_setup(const VolDev *, int, const FrameParams &, VolFrame *, unsigned *, cudaStream_t,
                               VisList *);
cudaError_t launch_brick_list(const VolDev *, int, const VolFrame *, const FrameParams &, long long,
                              long long, uint2 *, unsigned *, int, cudaStream_t, const VisList *,
                              const unsigned *, const unsigned *, uint2 *, long long);
cudaError_t launch_depth_max(const float *, const FrameParams &, unsigned *, int, cudaStream_t, unsigned *);
cudaError_t launch_integrate(const VolDev *, const VolFrame *, const uint2 *, const unsigned *,
                             const FrameParams &, const float *, const uint8_t *, Stats *, int,
                             cudaStream_t, uint2 *, unsigned *, unsigned);
cudaError_t launch_brick_flags(const VolDev &, int, cudaStream_t);
cudaError_t launch_mask_rebuild(const VolDev &, int, cudaStream_t);
cudaError_t launch_cell_flags(const VolDev *, const uint2 *, const unsigned *, int, cudaStream_t);
cudaError_t launch_cell_masks(const VolDev *, const uint2 *, const unsigned *, unsigned, int, cudaStream_t);
cudaError_t launch_raycast(const VolDev *, const VolFrame *, int, const FrameParams &, float *,
                           float *, uint8_t *, float *, int *, int, Stats *, int, cudaStream_t,
                           const VisList *);
cudaError_t launch_raycast_batch(const VolDev *, const VolFrame *, int, const FrameParams *, int, int, int,
                                 float *, float *, uint8_t *, float *, int *, Stats *, int, cudaStream_t,
                                 const VisList *);
int integrate_occupancy_grid(int num_sms);
int integrate_max_ctas_per_sm();
cudaError_t launch_raycast_backward(const BackwardArgs &A, cudaStream_t s);
size_t backward_ctas_per_pose(int width, int height);
cudaError_t launch_l1_stats(const float *, const float *, const uint8_t *, const uint8_t *, long long, float,
                            unsigned *, float *, cudaStream_t);
cudaError_t launch_gather_box(const void *src, int elem_bytes, const int nb[3], const int lo[3], const int n[3],
                              void *dst, int num_sms, cudaStream_t s);
cudaError_t launch_extract(const VolDev &, float *, uint8_t *, unsigned long long *, unsigned long long,
                           unsigned long long *, int, cudaStream_t);
cudaError_t launch_depth_maps(const float *, const mv_intrinsics &, float, float, const double *, float *, float *,
                              cudaStream_t);
cudaError_t launch_icp_system(const float *, const float *, const mv_intrinsics &, const double *, const float *,
                              const float *, const double *, float, float, float *, int, cudaStream_t);
int icp_grid(int num_sms);
cudaError_t launch_icp_step(const float *vertex, const float *normal, const mv_intrinsics &K, double *T_dev,
                            double *sys_dev, int *state_dev, const float *mvertex, const float *mnormal,
                            const double *T_model, float dist, float cos_min, float *partials, int grid,
                            cudaStream_t s);
cudaError_t launch_stream_gather(const VolDev &, const VolFrame *, const FrameParams &, const void *, const void *,
                                 unsigned long long *, int, cudaStream_t);
cudaError_t launch_stream_scatter(const VolDev &, const uint2 *, const unsigned *, void *, void *,
                                  unsigned long long *, int, cudaStream_t);
constexpr int kIcpTerms = 29;
cudaError_t graph_integrate(cudaGraph_t, cudaGraphExec_t, cudaGraphNode_t[6], cudaGraphNode_t,
                            const VolDev *, int, VolFrame *, const FrameParams &, long long, long long, uint2 *,
                            uint2 *, unsigned *, const float *, const uint8_t *, Stats *, int, int, VisList *,
                            uint2 *, unsigned, unsigned *);
cudaError_t graph_raycast(cudaGraph_t, cudaGraphExec_t, cudaGraphNode_t *, cudaGraphNode_t,
                          const VolDev *, int, VolFrame *, const FrameParams &, float *, float *, uint8_t *,
                          float *, int *, Stats *, int, VisList *);
}  // namespace mv

using namespace mv;

namespace {

struct Volume {
    int id = -1;
    mv_volume_desc desc{};
    int nb[3] = {0, 0, 0};
    int nsb[3] = {0, 0, 0};
    long long nbricks = 0, nsuper = 0;
    size_t fw_bytes = 0, rgba_bytes = 0, flag_bytes = 0;
    void *d_fw = nullptr;
    uint32_t *d_rgba = nullptr;
    uint8_t *d_flag = nullptr;
    void *d_mask = nullptr;  // voxel + cell masks while resident (derived, never swapped)
    void *h_fw = nullptr;
    uint32_t *h_rgba = nullptr;
    uint8_t *h_flag = nullptr;
    bool resident = false;
    cudaEvent_t ready = nullptr;  // allocation / swap-in copy finished
    bool ready_pending = false;
};

size_t fw_elem_bytes(int fmt) { return fmt == MV_TSDF_F32 ? 8 : 4; }

}  // namespace

struct mv_ctx {
    mv_config cfg{};
    int device = 0;
    int num_sms = 0;
    int grid_integrate = 0;
    int ray_tile = 0;
    int ctas_per_sm = 0;
    std::map<int, Volume *> vols;
    int next_id = 0;
    unsigned integrations = 0;  // id of the last integration call (brick listing stamps)
    cudaStream_t swap_stream = nullptr;
    cudaEvent_t last_event = nullptr;
    bool last_recorded = false;
    // device table of resident volumes (sorted by id)
    std::vector<VolDev> table;
    std::vector<int> table_ids;
    bool table_dirty = true;
    unsigned long long table_version = 0;
    // per-frame CUDA graph (mv_frame): rebuilt when its shape changes,
    // otherwise only its kernel-node parameters are updated
    struct FrameGraph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t nodes[7] = {};
        unsigned long long table_version = ~0ull;
        int width = 0, height = 0, grid_int = 0, tile = 0;
        bool two_level = false;
    } fg;
    VolDev *d_table = nullptr;
    VolFrame *d_vf = nullptr;
    uint2 *d_list = nullptr;
    size_t list_cap = 0;  // entries
    uint2 *d_slist = nullptr;  // super bricks in view (two-level work list)
    size_t slist_cap = 0;      // entries
    long long total_sup = 0;   // super bricks of the resident volumes
    long long resident_bricks = 0;  // bricks of the resident volumes
    int list_levels = 0;            // mv_tuning::work_list_levels
    unsigned *d_counter = nullptr;
    Stats *d_stats = nullptr;
    VisList *d_vis = nullptr;  // volumes in view of the current batched call
    unsigned *d_pyr = nullptr;  // depth-tile pyramid of the current frame
    size_t pyr_words = 0;
    unsigned long long *d_points = nullptr;  // point count of mv_extract_points
    mv::PinnedPool *pool = nullptr;          // pinned host buffers of swapped-out volumes
    // tracking scratch: the frame's vertex / normal maps, per-CTA ICP partials
    float *d_trk_v = nullptr, *d_trk_n = nullptr;
    size_t trk_px = 0;
    float *d_trk_part = nullptr;
    double *d_trk_loop = nullptr;  // mv_track's device loop: pose (16), system (44), then 2 ints of state
    // full-cover streaming (mv_frame_streamed): device staging slots that the
    // swapped-out volumes pass through, one copy stream per direction
    struct Slots {
        int n = 0;
        size_t fw_cap = 0, rgba_cap = 0, flag_cap = 0;  // bytes per slot
        long long list_cap = 0;                         // work-list entries
        void *fw[kMaxStreamSlots] = {};
        uint32_t *rgba[kMaxStreamSlots] = {};
        uint8_t *flag[kMaxStreamSlots] = {};
        VolDev *d_vol = nullptr;   // one descriptor per slot
        VolFrame *d_vf = nullptr;  // one camera-constant record per slot
        uint2 *list[kMaxStreamSlots] = {};  // per slot: the integration's work list
        unsigned *counter = nullptr;        // 4 per slot
        cudaStream_t h2d = nullptr, d2h = nullptr;
        cudaEvent_t loaded[kMaxStreamSlots] = {}, done[kMaxStreamSlots] = {}, freed[kMaxStreamSlots] = {};
        bool freed_rec[kMaxStreamSlots] = {};
    } ss;
    // mv_frame_host: two device buffer sets (frame in, maps out) and one
    // stream per pipeline stage; ticket t uses set t % 2
    struct HostPipe {
        cudaStream_t up = nullptr, run = nullptr, down = nullptr;
        int width = 0, height = 0;
        float *depth[2] = {}, *dout[2] = {}, *normal[2] = {}, *vertex[2] = {};
        uint8_t *rgb[2] = {}, *rgba[2] = {};
        int32_t *vid[2] = {};
        cudaEvent_t uploaded[2] = {}, computed[2] = {}, downloaded[2] = {};
        bool used[2] = {false, false};
        uint64_t next = 0;  // tickets issued
    } hp;
    // mv_raycast_batch: per view its parameters, camera constants of every
    // table slot and view list (capacity in views)
    FrameParams *d_pb = nullptr;
    VolFrame *d_vfb = nullptr;
    VisList *d_visb = nullptr;
    int batch_cap = 0;
    std::vector<FrameParams> h_pb;
    // pinned staging for the small per-call uploads (poses, view parameters,
    // gradient pointers): a copy from pageable memory would first wait for
    // the stream's earlier work; slot k is reused once its copy has run
    struct Stage {
        void *h = nullptr;
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
        bool recorded = false;
    } stage[4];
    int stage_next = 0;
    // raycast backward: per-slot gradient pointers and the poses of one call
    float **d_grad_ptrs = nullptr;
    float *d_poses = nullptr;  // per pose R, t (float) and per pose and slot the camera in voxels
    size_t poses_cap = 0;      // floats
    std::vector<float> h_pose_f;
    float *d_bw_partial = nullptr;  // per-CTA partial sums of the pose gradient
    size_t bw_partial_cap = 0;      // floats
    unsigned *d_l1 = nullptr;       // L1 loss statistics (kL1ScratchBytes), zeroed once
    // per-kernel launch counts and optional event timing
    bool timing = false;
    struct Timed { int kind; cudaEvent_t a, b; };
    std::vector<Timed> timed_pending;
    std::vector<cudaEvent_t> event_pool;
    uint64_t launches[MV_KERNEL_KINDS] = {};
    double ms[MV_KERNEL_KINDS] = {};
    uint64_t timed[MV_KERNEL_KINDS] = {};
    std::string err;
};

namespace mv {

// Method parameters every entry point accepts (mv_create and
// mv_integrate_noalloc alike).
bool valid_config(const mv_config &c)
{
    return c.trunc_voxels > 0.f && std::isfinite(c.trunc_voxels) && c.w_max >= 1.f &&
           c.w_max <= 1e30f && c.color_w_max >= 1 && c.color_w_max <= 255 && c.z_min >= 0.f &&
           c.z_max > c.z_min && c.ray_step >= 1.0f / 64.0f && c.ray_step <= 1.f && c.n_bisect >= 0 &&
           c.n_bisect <= 64;
}

}  // namespace mv

namespace {

mv_status fail(mv_ctx *c, mv_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

mv_status cuda_fail(mv_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? MV_ERR_OOM : MV_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define MV_CUDA(c, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

FrameParams make_params(const mv_ctx *c, const mv_intrinsics *K, const double T[16])
{
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
    P.z_min = c->cfg.z_min; P.z_max = c->cfg.z_max;
    P.trunc_vox = c->cfg.trunc_voxels;
    P.w_max = c->cfg.w_max;
    P.color_w_max = c->cfg.color_w_max;
    P.ray_step = c->cfg.ray_step;
    P.n_bisect = c->cfg.n_bisect;
    return P;
}

const double kIdentity[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};

bool valid_frame(const mv_intrinsics *K, const double *T)
{
    if (!K || !T) return false;
    if (K->width <= 0 || K->height <= 0 || K->width > 16384 || K->height > 16384) return false;
    if (!(K->fx > 0.f) || !(K->fy > 0.f) || !std::isfinite(K->fx) || !std::isfinite(K->fy) ||
        !std::isfinite(K->cx) || !std::isfinite(K->cy))
        return false;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T[i])) return false;
    return true;
}

VolDev make_voldev(const Volume &v)
{
    VolDev d{};
    d.fw = v.d_fw;
    d.rgba = v.d_rgba;
    d.bflag = v.d_flag;
    d.cflag = v.d_flag ? v.d_flag + cflag_offset(v.nbricks) : nullptr;
    d.surf = v.d_flag ? reinterpret_cast<unsigned *>(v.d_flag + flag_count_offset(v.nbricks)) : nullptr;
    d.sup = v.d_flag ? reinterpret_cast<unsigned *>(v.d_flag + super_offset(v.nbricks)) : nullptr;
    d.vmask = v.d_mask ? reinterpret_cast<unsigned long long *>(v.d_mask) : nullptr;
    d.cmask = v.d_mask ? reinterpret_cast<ulonglong2 *>(reinterpret_cast<uint8_t *>(v.d_mask) +
                                                         (size_t)v.nbricks * 128)
                       : nullptr;
    d.stamp = v.d_mask ? reinterpret_cast<unsigned *>(reinterpret_cast<uint8_t *>(v.d_mask) +
                                                      (size_t)v.nbricks * 256)
                       : nullptr;
    for (int a = 0; a < 3; ++a) d.nsb[a] = v.nsb[a];
    for (int a = 0; a < 3; ++a) {
        d.h[a] = v.desc.h_t[a];
        d.r[a] = v.desc.h_r[a];
        d.nb[a] = v.nb[a];
    }
    d.s = v.desc.voxel_size;
    d.inv_s = 1.0f / v.desc.voxel_size;
    d.fmt = v.desc.fmt;
    d.id = v.id;
    d.nbricks = v.nbricks;
    return d;
}

// Order this call after the previous call and after the pending copies of
// the resident volumes it reads (all of them, or only volume `only_id`);
// copies of volumes the call does not read keep running alongside.  Refresh
// the device table when the resident set changed.
mv_status begin_call(mv_ctx *c, cudaStream_t s, int only_id = -1)
{
    if (c->last_recorded) MV_CUDA(c, cudaStreamWaitEvent(s, c->last_event, 0));
    for (auto &kv : c->vols) {
        Volume *v = kv.second;
        if (!v->ready_pending) continue;
        if (cudaEventQuery(v->ready) == cudaSuccess) {
            v->ready_pending = false;
            continue;
        }
        if (!v->resident || (only_id >= 0 && v->id != only_id)) continue;
        MV_CUDA(c, cudaStreamWaitEvent(s, v->ready, 0));
    }
    if (c->table_dirty) {
        c->table.clear();
        c->table_ids.clear();
        long long base = 0, sbase = 0;
        for (auto &kv : c->vols) {
            Volume *v = kv.second;
            if (!v->resident) continue;
            VolDev d = make_voldev(*v);
            d.brick_base = base;
            base += v->nbricks;
            sbase += v->nsuper;
            c->table.push_back(d);
            c->table_ids.push_back(v->id);
        }
        if (!c->table.empty())
            MV_CUDA(c, cudaMemcpyAsync(c->d_table, c->table.data(), c->table.size() * sizeof(VolDev),
                                       cudaMemcpyHostToDevice, s));
        // the work list holds at most one entry per resident brick; the list of
        // bricks whose voxel masks changed follows it in the same buffer
        if ((size_t)base > c->list_cap) {
            if (c->d_list) MV_CUDA(c, cudaFreeAsync(c->d_list, s));
            c->d_list = nullptr;
            c->list_cap = 0;
            MV_CUDA(c, cudaMallocAsync((void **)&c->d_list, 2 * (size_t)base * sizeof(uint2), s));
            c->list_cap = (size_t)base;
        }
        // the super bricks in view: at most one entry per resident super brick
        if ((size_t)sbase > c->slist_cap) {
            if (c->d_slist) MV_CUDA(c, cudaFreeAsync(c->d_slist, s));
            c->d_slist = nullptr;
            c->slist_cap = 0;
            MV_CUDA(c, cudaMallocAsync((void **)&c->d_slist, (size_t)sbase * sizeof(uint2), s));
            c->slist_cap = (size_t)sbase;
        }
        c->total_sup = sbase;
        c->resident_bricks = base;
        c->table_dirty = false;
        c->table_version += 1;
    }
    return MV_OK;
}

// The batched calls build their work list in two levels (super bricks in
// view, then their bricks) when so tuned, or automatically from
// kTwoLevelBricks resident bricks on.
bool two_level_list(const mv_ctx *c)
{
    return c->list_levels == 2 || (c->list_levels == 0 && c->resident_bricks >= kTwoLevelBricks);
}

mv_status end_call(mv_ctx *c, cudaStream_t s)
{
    MV_CUDA(c, cudaEventRecord(c->last_event, s));
    c->last_recorded = true;
    return MV_OK;
}

cudaEvent_t pool_event(mv_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch one kernel (a callable returning cudaError_t), counting it and, when
// timing is on, bracketing it with events on its stream.
template <typename F>
cudaError_t counted_launch(mv_ctx *c, int kind, cudaStream_t s, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->timing) {
        a = pool_event(c);
        b = pool_event(c);
        if (a && b) cudaEventRecord(a, s);
    }
    cudaError_t e = launch();
    c->launches[kind] += 1;
    if (a && b) {
        cudaEventRecord(b, s);
        c->timed_pending.push_back({kind, a, b});
    } else {
        if (a) c->event_pool.push_back(a);
        if (b) c->event_pool.push_back(b);
    }
    return e;
}

mv_status collect_timings(mv_ctx *c)
{
    for (auto &t : c->timed_pending) {
        MV_CUDA(c, cudaEventSynchronize(t.b));
        float ms = 0.f;
        MV_CUDA(c, cudaEventElapsedTime(&ms, t.a, t.b));
        c->ms[t.kind] += ms;
        c->timed[t.kind] += 1;
        c->event_pool.push_back(t.a);
        c->event_pool.push_back(t.b);
    }
    c->timed_pending.clear();
    return MV_OK;
}

int table_slot(const mv_ctx *c, int id)
{
    auto it = std::lower_bound(c->table_ids.begin(), c->table_ids.end(), id);
    if (it == c->table_ids.end() || *it != id) return -1;
    return (int)(it - c->table_ids.begin());
}

mv_status find_volume(mv_ctx *c, int32_t id, Volume **out)
{
    auto it = c->vols.find(id);
    if (it == c->vols.end()) return fail(c, MV_ERR_NOT_FOUND, "no volume with id " + std::to_string(id));
    *out = it->second;
    return MV_OK;
}

mv_status wait_all(mv_ctx *c)
{
    if (c->last_recorded) MV_CUDA(c, cudaEventSynchronize(c->last_event));
    MV_CUDA(c, cudaStreamSynchronize(c->swap_stream));
    return MV_OK;
}

// brick-major <-> linear conversion on the host
template <typename T>
void bricks_to_linear(const Volume &v, const T *src, T *dst)
{
    const int rx = v.desc.h_r[0], ry = v.desc.h_r[1], rz = v.desc.h_r[2];
    for (int z = 0; z < rz; ++z)
        for (int y = 0; y < ry; ++y) {
            const long long rowb = ((long long)(z >> 3) * v.nb[1] + (y >> 3)) * v.nb[0];
            const int inner = ((z & 7) << 6) | ((y & 7) << 3);
            T *d = dst + ((size_t)z * ry + y) * rx;
            for (int x = 0; x < rx; ++x)
                d[x] = src[(rowb + (x >> 3)) * kBrickVox + inner + (x & 7)];
        }
}

template <typename T>
void linear_to_bricks(const Volume &v, const T *src, T *dst)
{
    const int rx = v.desc.h_r[0], ry = v.desc.h_r[1], rz = v.desc.h_r[2];
    for (int z = 0; z < rz; ++z)
        for (int y = 0; y < ry; ++y) {
            const long long rowb = ((long long)(z >> 3) * v.nb[1] + (y >> 3)) * v.nb[0];
            const int inner = ((z & 7) << 6) | ((y & 7) << 3);
            const T *s = src + ((size_t)z * ry + y) * rx;
            for (int x = 0; x < rx; ++x)
                dst[(rowb + (x >> 3)) * kBrickVox + inner + (x & 7)] = s[x];
        }
}

void free_host(mv_ctx *c, Volume *v)
{
    c->pool->give(v->h_fw, v->fw_bytes);
    c->pool->give(v->h_rgba, v->rgba_bytes);
    c->pool->give(v->h_flag, v->flag_bytes);
    v->h_fw = nullptr;
    v->h_rgba = nullptr;
    v->h_flag = nullptr;
}

}  // namespace


// ---------------------------------------------------------------------------
// full-cover streaming
// ---------------------------------------------------------------------------
namespace {

__global__ void put_voldev_kernel(VolDev v, VolDev *dst)
{
    if (threadIdx.x == 0) *dst = v;
}

// (Re)allocate the staging slots for n slots of at least the given sizes.
mv_status ensure_slots(mv_ctx *c, int n, size_t fw, size_t rgba, size_t flag, long long bricks,
                       cudaStream_t s)
{
    auto &ss = c->ss;
    if (!ss.h2d) MV_CUDA(c, cudaStreamCreateWithFlags(&ss.h2d, cudaStreamNonBlocking));
    if (!ss.d2h) MV_CUDA(c, cudaStreamCreateWithFlags(&ss.d2h, cudaStreamNonBlocking));
    if (!ss.d_vol) MV_CUDA(c, cudaMalloc((void **)&ss.d_vol, sizeof(VolDev) * kMaxStreamSlots));
    if (!ss.d_vf) MV_CUDA(c, cudaMalloc((void **)&ss.d_vf, sizeof(VolFrame) * kMaxStreamSlots));
    if (!ss.counter) MV_CUDA(c, cudaMalloc((void **)&ss.counter, sizeof(unsigned) * 4 * kMaxStreamSlots));
    for (int j = 0; j < kMaxStreamSlots; ++j) {
        if (!ss.loaded[j]) MV_CUDA(c, cudaEventCreateWithFlags(&ss.loaded[j], cudaEventDisableTiming));
        if (!ss.done[j]) MV_CUDA(c, cudaEventCreateWithFlags(&ss.done[j], cudaEventDisableTiming));
        if (!ss.freed[j]) MV_CUDA(c, cudaEventCreateWithFlags(&ss.freed[j], cudaEventDisableTiming));
    }
    const bool grow = n > ss.n || fw > ss.fw_cap || rgba > ss.rgba_cap || flag > ss.flag_cap ||
                      bricks > ss.list_cap;
    if (!grow) return MV_OK;
    // slots in use by earlier calls are released in stream order
    for (int j = 0; j < ss.n; ++j)
        if (ss.freed_rec[j]) MV_CUDA(c, cudaStreamWaitEvent(s, ss.freed[j], 0));
    for (int j = 0; j < kMaxStreamSlots; ++j) {
        if (ss.fw[j]) MV_CUDA(c, cudaFreeAsync(ss.fw[j], s));
        if (ss.rgba[j]) MV_CUDA(c, cudaFreeAsync(ss.rgba[j], s));
        if (ss.flag[j]) MV_CUDA(c, cudaFreeAsync(ss.flag[j], s));
        if (ss.list[j]) MV_CUDA(c, cudaFreeAsync(ss.list[j], s));
        ss.fw[j] = nullptr;
        ss.rgba[j] = nullptr;
        ss.flag[j] = nullptr;
        ss.list[j] = nullptr;
        ss.freed_rec[j] = false;
    }
    ss.n = 0;
    ss.fw_cap = std::max(fw, ss.fw_cap);
    ss.rgba_cap = std::max(rgba, ss.rgba_cap);
    ss.flag_cap = std::max(flag, ss.flag_cap);
    ss.list_cap = std::max(bricks, ss.list_cap);
    n = std::max(n, 1);
    for (int j = 0; j < n; ++j) {
        MV_CUDA(c, cudaMallocAsync(&ss.fw[j], ss.fw_cap, s));
        MV_CUDA(c, cudaMallocAsync((void **)&ss.rgba[j], ss.rgba_cap, s));
        MV_CUDA(c, cudaMallocAsync((void **)&ss.flag[j], ss.flag_cap, s));
        MV_CUDA(c, cudaMallocAsync((void **)&ss.list[j], sizeof(uint2) * (size_t)ss.list_cap, s));
    }
    ss.n = n;
    return MV_OK;
}

void free_slots(mv_ctx *c, cudaStream_t s)
{
    auto &ss = c->ss;
    for (int j = 0; j < kMaxStreamSlots; ++j) {
        if (ss.fw[j]) cudaFreeAsync(ss.fw[j], s);
        if (ss.rgba[j]) cudaFreeAsync(ss.rgba[j], s);
        if (ss.flag[j]) cudaFreeAsync(ss.flag[j], s);
        if (ss.loaded[j]) cudaEventDestroy(ss.loaded[j]);
        if (ss.done[j]) cudaEventDestroy(ss.done[j]);
        if (ss.freed[j]) cudaEventDestroy(ss.freed[j]);
    }
    for (int j = 0; j < kMaxStreamSlots; ++j)
        if (ss.list[j]) cudaFreeAsync(ss.list[j], s);
    if (ss.d_vol) cudaFree(ss.d_vol);
    if (ss.d_vf) cudaFree(ss.d_vf);
    if (ss.counter) cudaFree(ss.counter);
    if (ss.h2d) cudaStreamDestroy(ss.h2d);
    if (ss.d2h) cudaStreamDestroy(ss.d2h);
    ss = mv_ctx::Slots{};
}

}  // namespace

namespace {

// Device buffers and events of the host pipeline (after a full synchronise).
void free_host_pipe(mv_ctx *c)
{
    auto &hp = c->hp;
    for (int b = 0; b < 2; ++b) {
        cudaFree(hp.depth[b]);
        cudaFree(hp.rgb[b]);
        cudaFree(hp.dout[b]);
        cudaFree(hp.normal[b]);
        cudaFree(hp.rgba[b]);
        cudaFree(hp.vertex[b]);
        cudaFree(hp.vid[b]);
        hp.depth[b] = hp.dout[b] = hp.normal[b] = hp.vertex[b] = nullptr;
        hp.rgb[b] = hp.rgba[b] = nullptr;
        hp.vid[b] = nullptr;
        hp.used[b] = false;
    }
    hp.width = hp.height = 0;
}

// Allocate the pipeline's streams, events and the two buffer sets for w x h
// frames (once, and again when the image size changes).
cudaError_t ensure_host_pipe(mv_ctx *c, int w, int h)
{
    auto &hp = c->hp;
    cudaError_t e = cudaSuccess;
    if (!hp.up) {
        for (cudaStream_t *st : {&hp.up, &hp.run, &hp.down})
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b)
            for (cudaEvent_t *ev : {&hp.uploaded[b], &hp.computed[b], &hp.downloaded[b]})
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    if (hp.width == w && hp.height == h) return cudaSuccess;
    // the buffers of earlier frames may still be in use
    for (cudaStream_t st : {hp.up, hp.run, hp.down}) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
    }
    free_host_pipe(c);
    const size_t n = (size_t)w * (size_t)h;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc((void **)&hp.depth[b], n * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&hp.rgb[b], n * 3);
        if (e == cudaSuccess) e = cudaMalloc((void **)&hp.dout[b], n * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&hp.normal[b], n * 12);
        if (e == cudaSuccess) e = cudaMalloc((void **)&hp.rgba[b], n * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&hp.vertex[b], n * 12);
        if (e == cudaSuccess) e = cudaMalloc((void **)&hp.vid[b], n * 4);
    }
    if (e != cudaSuccess) {
        free_host_pipe(c);
        return e;
    }
    hp.width = w;
    hp.height = h;
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char *mv_version(void) { return "mvtsdf 0.1.0 (sm_103a)"; }

mv_status mv_config_default(mv_config *out)
{
    if (!out) return MV_ERR_ARG;
    out->trunc_voxels = 4.0f;
    out->w_max = 128.0f;
    out->color_w_max = 255;
    out->z_min = 0.0f;
    out->z_max = INFINITY;
    out->ray_step = 1.0f;
    out->n_bisect = 8;
    return MV_OK;
}

mv_status mv_create(const mv_config *cfg, int32_t device, mv_ctx **out)
{
    if (!out) return MV_ERR_ARG;
    *out = nullptr;
    mv_config c;
    if (cfg) c = *cfg; else mv_config_default(&c);
    if (!valid_config(c)) return MV_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MV_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return MV_ERR_CUDA;
    mv_ctx *x = new mv_ctx();
    x->cfg = c;
    x->device = device;
    x->pool = new mv::PinnedPool();
    cudaError_t e = cudaDeviceGetAttribute(&x->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x->swap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->last_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void **)&x->d_table, sizeof(VolDev) * kMaxVolumes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&x->d_vf, sizeof(VolFrame) * kMaxVolumes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&x->d_counter, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&x->d_stats, sizeof(Stats));
    if (e == cudaSuccess) e = cudaMalloc((void **)&x->d_vis, sizeof(VisList));
    if (e == cudaSuccess) e = cudaMalloc((void **)&x->d_grad_ptrs, sizeof(float *) * kMaxVolumes);
    if (e == cudaSuccess) e = cudaMemset(x->d_stats, 0, sizeof(Stats));
    if (e != cudaSuccess) {
        mv_destroy(x);
        return e == cudaErrorMemoryAllocation ? MV_ERR_OOM : MV_ERR_CUDA;
    }
    x->ctas_per_sm = integrate_max_ctas_per_sm();
    x->grid_integrate = x->num_sms * x->ctas_per_sm;
    *out = x;
    return MV_OK;
}

mv_status mv_destroy(mv_ctx *c)
{
    if (!c) return MV_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    // stream-ordered allocations go back through the stream-ordered allocator
    cudaStream_t s = c->swap_stream;
    for (auto &kv : c->vols) {
        Volume *v = kv.second;
        if (v->d_fw) cudaFreeAsync(v->d_fw, s);
        if (v->d_rgba) cudaFreeAsync(v->d_rgba, s);
        if (v->d_flag) cudaFreeAsync(v->d_flag, s);
        if (v->d_mask) cudaFreeAsync(v->d_mask, s);
    }
    if (c->d_list) cudaFreeAsync(c->d_list, s);
    if (c->d_slist) cudaFreeAsync(c->d_slist, s);
    free_slots(c, s);
    if (s) cudaStreamSynchronize(s);
    for (auto &kv : c->vols) {
        Volume *v = kv.second;
        free_host(c, v);
        if (v->ready) cudaEventDestroy(v->ready);
        delete v;
    }
    if (c->d_table) cudaFree(c->d_table);
    if (c->d_vf) cudaFree(c->d_vf);
    if (c->d_counter) cudaFree(c->d_counter);
    if (c->d_stats) cudaFree(c->d_stats);
    if (c->d_vis) cudaFree(c->d_vis);
    if (c->d_pyr) cudaFree(c->d_pyr);
    if (c->d_points) cudaFree(c->d_points);
    if (c->d_trk_v) cudaFree(c->d_trk_v);
    if (c->d_trk_n) cudaFree(c->d_trk_n);
    if (c->d_trk_part) cudaFree(c->d_trk_part);
    if (c->d_trk_loop) cudaFree(c->d_trk_loop);
    if (c->d_grad_ptrs) cudaFree(c->d_grad_ptrs);
    if (c->fg.exec) cudaGraphExecDestroy(c->fg.exec);
    if (c->fg.g) cudaGraphDestroy(c->fg.g);
    if (c->d_poses) cudaFree(c->d_poses);
    if (c->d_bw_partial) cudaFree(c->d_bw_partial);
    if (c->d_l1) cudaFree(c->d_l1);
    for (auto &st : c->stage) {
        if (st.h) cudaFreeHost(st.h);
        if (st.ev) cudaEventDestroy(st.ev);
    }
    free_host_pipe(c);
    if (c->d_pb) cudaFree(c->d_pb);
    if (c->d_vfb) cudaFree(c->d_vfb);
    if (c->d_visb) cudaFree(c->d_visb);
    for (cudaStream_t st : {c->hp.up, c->hp.run, c->hp.down})
        if (st) cudaStreamDestroy(st);
    for (int b = 0; b < 2; ++b)
        for (cudaEvent_t ev : {c->hp.uploaded[b], c->hp.computed[b], c->hp.downloaded[b]})
            if (ev) cudaEventDestroy(ev);
    for (auto &t : c->timed_pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->last_event) cudaEventDestroy(c->last_event);
    if (c->swap_stream) cudaStreamDestroy(c->swap_stream);
    delete c->pool;  // after the volumes gave their host buffers back
    delete c;
    return MV_OK;
}

mv_status mv_extract_points(mv_ctx *c, int32_t id, float *xyz, uint8_t *rgb, uint64_t *edge, uint64_t cap,
                            uint64_t *n, void *stream)
{
    if (!c || !n) return fail(c, MV_ERR_ARG, "null argument");
    if (!aligned_to({xyz}, 4) || !aligned_to({edge}, 8))
        return fail(c, MV_ERR_ARG, "xyz must be 4-byte and edge 8-byte aligned");
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    if (!v->resident) return fail(c, MV_ERR_NOT_RESIDENT, "volume is swapped out");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    st = begin_call(c, s, id);
    if (st) return st;
    if (!c->d_points) MV_CUDA(c, cudaMalloc((void **)&c->d_points, sizeof(unsigned long long)));
    MV_CUDA(c, cudaMemsetAsync(c->d_points, 0, sizeof(unsigned long long), s));
    const VolDev d = make_voldev(*v);
    MV_CUDA(c, counted_launch(c, MV_KERNEL_EXTRACT, s, [&] {
        return launch_extract(d, xyz, rgb, reinterpret_cast<unsigned long long *>(edge), cap, c->d_points,
                              c->num_sms, s); }));
    unsigned long long count = 0;
    MV_CUDA(c, cudaMemcpyAsync(&count, c->d_points, sizeof(count), cudaMemcpyDeviceToHost, s));
    MV_CUDA(c, cudaStreamSynchronize(s));
    *n = count;
    st = end_call(c, s);
    if (st) return st;
    return count > cap ? fail(c, MV_ERR_CAPACITY, "more points than cap") : MV_OK;
}

static mv_status track_scratch(mv_ctx *c, const mv_intrinsics *K, cudaStream_t s)
{
    const size_t px = (size_t)K->width * K->height;
    if (px > c->trk_px) {
        if (c->d_trk_v) MV_CUDA(c, cudaFreeAsync(c->d_trk_v, s));
        if (c->d_trk_n) MV_CUDA(c, cudaFreeAsync(c->d_trk_n, s));
        c->d_trk_v = c->d_trk_n = nullptr;
        c->trk_px = 0;
        MV_CUDA(c, cudaMallocAsync((void **)&c->d_trk_v, 3 * sizeof(float) * px, s));
        MV_CUDA(c, cudaMallocAsync((void **)&c->d_trk_n, 3 * sizeof(float) * px, s));
        c->trk_px = px;
    }
    if (!c->d_trk_part)
        MV_CUDA(c, cudaMalloc((void **)&c->d_trk_part, sizeof(float) * kIcpTerms * icp_grid(c->num_sms)));
    if (!c->d_trk_loop) MV_CUDA(c, cudaMalloc((void **)&c->d_trk_loop, sizeof(double) * 61));
    return MV_OK;
}

// One ICP linearisation on device maps; the partials are added on the host
// in CTA order (deterministic).
static mv_status upload_small(mv_ctx *c, void *dst, const void *src, size_t bytes, cudaStream_t s);

static mv_status icp_linearise(mv_ctx *c, const float *v, const float *n, const mv_intrinsics *K,
                               const double T_est[16], const float *mv_, const float *mn, const double T_model[16],
                               const mv_icp_config *cfg, mv_icp_system *out, cudaStream_t s)
{
    const int grid = icp_grid(c->num_sms);
    MV_CUDA(c, counted_launch(c, MV_KERNEL_ICP, s, [&] {
        return launch_icp_system(v, n, *K, T_est, mv_, mn, T_model, cfg->dist, cfg->cos_min, c->d_trk_part, grid,
                                 s); }));
    std::vector<float> part((size_t)grid * kIcpTerms);
    MV_CUDA(c, cudaMemcpyAsync(part.data(), c->d_trk_part, sizeof(float) * part.size(), cudaMemcpyDeviceToHost, s));
    MV_CUDA(c, cudaStreamSynchronize(s));
    double sum[kIcpTerms] = {0};
    for (int g = 0; g < grid; ++g)
        for (int k = 0; k < kIcpTerms; ++k) sum[k] += (double)part[(size_t)g * kIcpTerms + k];
    int k = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++k) out->A[6 * i + j] = out->A[6 * j + i] = sum[k];
    for (int i = 0; i < 6; ++i) out->b[i] = sum[21 + i];
    out->error = sum[27];
    out->inliers = (int64_t)std::llround(sum[28]);
    return MV_OK;
}

static bool valid_icp(const mv_icp_config *cfg)
{
    return cfg && cfg->iterations >= 0 && cfg->iterations <= 1000 && cfg->dist > 0.f && std::isfinite(cfg->dist) &&
           cfg->cos_min >= -1.f && cfg->cos_min <= 1.f;
}

mv_status mv_depth_to_maps(mv_ctx *c, const float *depth, const mv_intrinsics *K, const double T[16],
                           float *vertex, float *normal, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!depth || !vertex || !normal || !valid_frame(K, T ? T : kIdentity))
        return fail(c, MV_ERR_ARG, "bad arguments");
    if (!aligned_to({depth, vertex, normal}, 4)) return fail(c, MV_ERR_ARG, "maps must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    MV_CUDA(c, counted_launch(c, MV_KERNEL_DEPTH_MAPS, s, [&] {
        return launch_depth_maps(depth, *K, c->cfg.z_min, c->cfg.z_max, T, vertex, normal, s); }));
    return MV_OK;
}

mv_status mv_icp_linearize(mv_ctx *c, const float *vertex, const float *normal, const mv_intrinsics *K,
                        const double T_est[16], const float *model_vertex, const float *model_normal,
                        const double T_model[16], const mv_icp_config *cfg, mv_icp_system *out, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!vertex || !normal || !model_vertex || !model_normal || !out || !valid_frame(K, T_est) ||
        !valid_frame(K, T_model) || !valid_icp(cfg))
        return fail(c, MV_ERR_ARG, "bad arguments");
    if (!aligned_to({vertex, normal, model_vertex, model_normal}, 4))
        return fail(c, MV_ERR_ARG, "maps must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    mv_status st = track_scratch(c, K, s);
    if (st) return st;
    return icp_linearise(c, vertex, normal, K, T_est, model_vertex, model_normal, T_model, cfg, out, s);
}

mv_status mv_track(mv_ctx *c, const float *depth, const mv_intrinsics *K, const float *model_vertex,
                   const float *model_normal, const double T_model[16], const double T_init[16],
                   const mv_icp_config *cfg, double T_out[16], mv_icp_system *last, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!depth || !model_vertex || !model_normal || !T_out || !valid_frame(K, T_model) ||
        !valid_frame(K, T_init) || !valid_icp(cfg))
        return fail(c, MV_ERR_ARG, "bad arguments");
    if (!aligned_to({depth, model_vertex, model_normal}, 4)) return fail(c, MV_ERR_ARG, "maps must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    mv_status st = track_scratch(c, K, s);
    if (st) return st;
    MV_CUDA(c, counted_launch(c, MV_KERNEL_DEPTH_MAPS, s, [&] {
        return launch_depth_maps(depth, *K, c->cfg.z_min, c->cfg.z_max, nullptr, c->d_trk_v, c->d_trk_n, s); }));
    // the Gauss-Newton loop on the device (no host round trip per step): the
    // pose and the last system stay in device memory and are read back once
    double *d_T = c->d_trk_loop, *d_sys = c->d_trk_loop + 16;
    int *d_state = reinterpret_cast<int *>(c->d_trk_loop + 60);
    st = upload_small(c, d_T, T_init, sizeof(double) * 16, s);
    if (st) return st;
    MV_CUDA(c, cudaMemsetAsync(d_sys, 0, sizeof(double) * 44 + sizeof(int) * 2, s));
    const int grid = icp_grid(c->num_sms);
    for (int it = 0; it < cfg->iterations; ++it)
        MV_CUDA(c, counted_launch(c, MV_KERNEL_ICP, s, [&] {
            return launch_icp_step(c->d_trk_v, c->d_trk_n, *K, d_T, d_sys, d_state, model_vertex, model_normal,
                                   T_model, cfg->dist, cfg->cos_min, c->d_trk_part, grid, s); }));
    double back[60];
    MV_CUDA(c, cudaMemcpyAsync(back, c->d_trk_loop, sizeof(back), cudaMemcpyDeviceToHost, s));
    MV_CUDA(c, cudaStreamSynchronize(s));
    for (int i = 0; i < 16; ++i) T_out[i] = back[i];
    if (last) {
        mv_icp_system sys{};
        for (int i = 0; i < 36; ++i) sys.A[i] = back[16 + i];
        for (int i = 0; i < 6; ++i) sys.b[i] = back[52 + i];
        sys.error = back[58];
        sys.inliers = (int64_t)std::llround(back[59]);
        *last = sys;
    }
    return MV_OK;
}

mv_status mv_reserve_host(mv_ctx *c, const mv_volume_desc *d, int32_t count)
{
    if (!c || !d || count < 0 || count > 4096) return fail(c, MV_ERR_ARG, "bad arguments");
    Volume shape;
    shape.desc = *d;
    shape.nbricks = 1;
    shape.nsuper = 1;
    for (int a = 0; a < 3; ++a) {
        if (d->h_r[a] < 2 || d->h_r[a] > 8192) return fail(c, MV_ERR_ARG, "bad volume size");
        shape.nb[a] = (d->h_r[a] + kBrick - 1) / kBrick;
        shape.nbricks *= shape.nb[a];
        shape.nsb[a] = (shape.nb[a] + kSuper - 1) / kSuper;
        shape.nsuper *= shape.nsb[a];
    }
    if (d->fmt < MV_TSDF_F32 || d->fmt > MV_TSDF_I16) return fail(c, MV_ERR_ARG, "bad format");
    cudaSetDevice(c->device);
    const bool ok = c->pool->reserve((size_t)shape.nbricks * kBrickVox * fw_elem_bytes(d->fmt), count) &&
                    c->pool->reserve((size_t)shape.nbricks * kBrickVox * 4, count) &&
                    c->pool->reserve(flag_alloc_bytes(shape.nbricks, shape.nsuper), count);
    return ok ? MV_OK : fail(c, MV_ERR_OOM, "pinned host allocation failed");
}

mv_status mv_get_config(const mv_ctx *c, mv_config *out)
{
    if (!c || !out) return MV_ERR_ARG;
    *out = c->cfg;
    return MV_OK;
}

int32_t mv_get_device(const mv_ctx *c)
{
    return c ? c->device : -1;
}

const char *mv_last_error(const mv_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

mv_status mv_add_volume(mv_ctx *c, const mv_volume_desc *d, int32_t *out_id)
{
    if (!c || !d || !out_id) return fail(c, MV_ERR_ARG, "null argument");
    for (int a = 0; a < 3; ++a)
        if (d->h_r[a] < 2 || d->h_r[a] > 8192) return fail(c, MV_ERR_ARG, "h_r must be in [2, 8192]");
    if (!(d->voxel_size > 0.f) || !std::isfinite(d->voxel_size)) return fail(c, MV_ERR_ARG, "voxel_size must be > 0");
    if (d->fmt < MV_TSDF_F32 || d->fmt > MV_TSDF_I16) return fail(c, MV_ERR_ARG, "bad storage format");
    if (d->fmt != MV_TSDF_F32 && c->cfg.w_max > 65535.f)
        return fail(c, MV_ERR_ARG, "w_max > 65535 does not fit a uint16 weight");
    if ((int)c->vols.size() >= kMaxVolumes) return fail(c, MV_ERR_CAPACITY, "too many volumes");
    cudaSetDevice(c->device);
    Volume *v = new Volume();
    v->desc = *d;
    v->nbricks = 1;
    v->nsuper = 1;
    for (int a = 0; a < 3; ++a) {
        v->nb[a] = (d->h_r[a] + kBrick - 1) / kBrick;
        v->nbricks *= v->nb[a];
        v->nsb[a] = (v->nb[a] + kSuper - 1) / kSuper;
        v->nsuper *= v->nsb[a];
    }
    v->fw_bytes = (size_t)v->nbricks * kBrickVox * fw_elem_bytes(d->fmt);
    v->rgba_bytes = (size_t)v->nbricks * kBrickVox * 4;
    v->flag_bytes = flag_alloc_bytes(v->nbricks, v->nsuper);  // brick, cell, count, super counts
    cudaStream_t s = c->swap_stream;
    cudaError_t e = cudaEventCreateWithFlags(&v->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocAsync(&v->d_fw, v->fw_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&v->d_rgba, v->rgba_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&v->d_flag, v->flag_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&v->d_mask, mask_alloc_bytes(v->nbricks), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->d_fw, 0, v->fw_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->d_mask, 0, mask_alloc_bytes(v->nbricks), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->d_rgba, 0, v->rgba_bytes, s);
    // nothing observed yet: every brick NONEG, every cell brick skipped, the
    // counts (bricks without NONEG, cell bricks without skip) all 0
    if (e == cudaSuccess) e = cudaMemsetAsync(v->d_flag, 0, v->flag_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->d_flag, kFlagsNew, (size_t)v->nbricks, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(v->d_flag + cflag_offset(v->nbricks), kCellSkip, (size_t)v->nbricks, s);
    if (e == cudaSuccess) e = cudaEventRecord(v->ready, s);
    if (e != cudaSuccess) {
        if (v->d_fw) cudaFreeAsync(v->d_fw, s);
        if (v->d_rgba) cudaFreeAsync(v->d_rgba, s);
        if (v->d_flag) cudaFreeAsync(v->d_flag, s);
        if (v->d_mask) cudaFreeAsync(v->d_mask, s);
        cudaStreamSynchronize(s);
        if (v->ready) cudaEventDestroy(v->ready);
        delete v;
        cudaGetLastError();
        return cuda_fail(c, e, "allocating volume storage");
    }
    v->ready_pending = true;
    v->resident = true;
    v->id = c->next_id++;
    c->vols[v->id] = v;
    c->table_dirty = true;
    *out_id = v->id;
    return MV_OK;
}

mv_status mv_remove_volume(mv_ctx *c, int32_t id)
{
    if (!c) return MV_ERR_ARG;
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    cudaSetDevice(c->device);
    cudaStream_t s = c->swap_stream;
    if (c->last_recorded) MV_CUDA(c, cudaStreamWaitEvent(s, c->last_event, 0));
    if (v->d_fw) MV_CUDA(c, cudaFreeAsync(v->d_fw, s));
    if (v->d_rgba) MV_CUDA(c, cudaFreeAsync(v->d_rgba, s));
    if (v->d_flag) MV_CUDA(c, cudaFreeAsync(v->d_flag, s));
    if (v->d_mask) MV_CUDA(c, cudaFreeAsync(v->d_mask, s));
    if (v->h_fw || v->h_rgba || v->h_flag) {
        MV_CUDA(c, cudaStreamSynchronize(s));  // in-flight copies may still read the host copy
        free_host(c, v);
    }
    if (v->ready) {
        cudaEventSynchronize(v->ready);
        cudaEventDestroy(v->ready);
    }
    c->vols.erase(id);
    delete v;
    c->table_dirty = true;
    return MV_OK;
}

mv_status mv_query(mv_ctx *c, int32_t id, mv_volume_info *out)
{
    if (!c || !out) return fail(c, MV_ERR_ARG, "null argument");
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    out->desc = v->desc;
    out->resident = v->resident ? 1 : 0;
    out->reserved = 0;
    const size_t tot = v->fw_bytes + v->rgba_bytes + v->flag_bytes;
    out->device_bytes = v->resident ? tot + mask_alloc_bytes(v->nbricks) : 0;
    out->host_bytes = v->h_fw ? tot : 0;
    return MV_OK;
}

mv_status mv_list_volumes(mv_ctx *c, int32_t *ids, int32_t cap, int32_t *count)
{
    if (!c || !count || (cap > 0 && !ids)) return fail(c, MV_ERR_ARG, "null argument");
    int n = 0;
    for (auto &kv : c->vols) {
        if (n < cap) ids[n] = kv.first;
        ++n;
    }
    *count = n;
    return MV_OK;
}

// The depth-tile pyramid buffer, grown to the frame size (before any graph
// or launch of the call uses it).
// Copy `bytes` of host data to device memory on stream s through the
// context's pinned staging ring (the source may be reused on return).
static mv_status upload_small(mv_ctx *c, void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    auto &st = c->stage[c->stage_next];
    c->stage_next = (c->stage_next + 1) % 4;
    if (!st.ev) MV_CUDA(c, cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming));
    if (st.recorded) MV_CUDA(c, cudaEventSynchronize(st.ev));  // its previous copy has run
    if (bytes > st.cap) {
        if (st.h) MV_CUDA(c, cudaFreeHost(st.h));
        st.h = nullptr;
        st.cap = 0;
        const size_t cap = bytes < 65536 ? 65536 : bytes;
        MV_CUDA(c, cudaMallocHost(&st.h, cap));
        st.cap = cap;
    }
    std::memcpy(st.h, src, bytes);
    MV_CUDA(c, cudaMemcpyAsync(dst, st.h, bytes, cudaMemcpyHostToDevice, s));
    MV_CUDA(c, cudaEventRecord(st.ev, s));
    st.recorded = true;
    return MV_OK;
}

static mv_status ensure_pyramid(mv_ctx *c, const mv_intrinsics *K)
{
    // the largest-depth pyramid, then the smallest-depth one
    const size_t words = 2 * (size_t)pyr_dims(K->width, K->height).off[kPyrLevels];
    if (words <= c->pyr_words) return MV_OK;
    MV_CUDA(c, cudaDeviceSynchronize());  // an earlier call may still read the old buffer
    if (c->d_pyr) MV_CUDA(c, cudaFree(c->d_pyr));
    c->d_pyr = nullptr;
    c->pyr_words = 0;
    MV_CUDA(c, cudaMalloc((void **)&c->d_pyr, words * sizeof(unsigned)));
    c->pyr_words = words;
    return MV_OK;
}

static mv_status integrate_impl(mv_ctx *c, int32_t only_id, const float *depth, const uint8_t *rgb,
                                const mv_intrinsics *K, const double T[16], void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!depth || !valid_frame(K, T)) return fail(c, MV_ERR_ARG, "bad frame arguments");
    if (!aligned_to({depth}, 4)) return fail(c, MV_ERR_ARG, "depth must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (only_id >= 0) {
        Volume *v;
        mv_status st = find_volume(c, only_id, &v);
        if (st) return st;
        if (!v->resident) return fail(c, MV_ERR_NOT_RESIDENT, "volume is swapped out");
    }
    mv_status st = begin_call(c, s, only_id);
    if (st) return st;
    if (c->table.empty()) return end_call(c, s);
    const FrameParams P = make_params(c, K, T);
    int slot0 = 0, nvol = (int)c->table.size();
    if (only_id >= 0) {
        slot0 = table_slot(c, only_id);
        nvol = 1;
    }
    const VolDev *tab = c->d_table + slot0;
    VolFrame *vf = c->d_vf + slot0;
    const long long gb0 = c->table[slot0].brick_base;
    const long long total = only_id >= 0 ? c->table[slot0].nbricks
                                         : c->table.back().brick_base + c->table.back().nbricks;
    VisList *vis = only_id >= 0 ? nullptr : c->d_vis;  // batched: only volumes in view
    const bool two_level = vis && two_level_list(c);
    st = ensure_pyramid(c, K);
    if (st) return st;
    const unsigned stamp = ++c->integrations;
    MV_CUDA(c, counted_launch(c, MV_KERNEL_SETUP, s, [&] {
        return launch_frame_setup(tab, nvol, P, vf, c->d_counter, s, vis); }));
    MV_CUDA(c, counted_launch(c, MV_KERNEL_DEPTH_MAX, s, [&] {
        return launch_depth_max(depth, P, c->d_counter + 1, c->num_sms, s, c->d_pyr); }));
    MV_CUDA(c, counted_launch(c, MV_KERNEL_BRICK_LIST, s, [&] {
        return launch_brick_list(tab, nvol, vf, P, gb0, total, c->d_list, c->d_counter, c->num_sms, s, vis,
                                 c->d_counter + 1, c->d_pyr, two_level ? c->d_slist : nullptr, c->total_sup); }));
    if (two_level) c->launches[MV_KERNEL_BRICK_LIST] += 1;  // the two-level list is two kernels
    // every resident volume keeps cell masks: the integration lists the bricks
    // whose voxel masks changed (second half of the work-list buffer) and the
    // refresh recomputes the cell masks and flags that read them
    uint2 *changed = c->d_list + c->list_cap;
    MV_CUDA(c, counted_launch(c, MV_KERNEL_INTEGRATE, s, [&] {
        return launch_integrate(tab, vf, c->d_list, c->d_counter, P, depth, rgb, c->d_stats,
                                c->grid_integrate, s, changed, c->d_counter + 2, stamp); }));
    MV_CUDA(c, counted_launch(c, MV_KERNEL_CELL_FLAGS, s, [&] {
        return launch_cell_masks(tab, changed, c->d_counter + 2, stamp, c->num_sms, s); }));
    return end_call(c, s);
}

mv_status mv_integrate(mv_ctx *c, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                       const double T[16], void *stream)
{
    return integrate_impl(c, -1, depth, rgb, K, T, stream);
}

mv_status mv_integrate_volume(mv_ctx *c, int32_t id, const float *depth, const uint8_t *rgb,
                              const mv_intrinsics *K, const double T[16], void *stream)
{
    if (id < 0) return fail(c, MV_ERR_NOT_FOUND, "negative id");
    return integrate_impl(c, id, depth, rgb, K, T, stream);
}

static mv_status raycast_impl(mv_ctx *c, int32_t only_id, int first, const mv_intrinsics *K,
                              const double T[16], float *depth, float *normal, uint8_t *rgba,
                              float *vertex, int32_t *vol_id, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!valid_frame(K, T)) return fail(c, MV_ERR_ARG, "bad view arguments");
    const bool merge = only_id >= 0 && !first;
    if (only_id >= 0 && (!depth || !vol_id))
        return fail(c, MV_ERR_ARG, "per-volume raycast needs depth and vol_id (merge state)");
    if (!aligned_to({depth, normal, rgba, vertex, vol_id}, 4))
        return fail(c, MV_ERR_ARG, "maps must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (only_id >= 0) {
        Volume *v;
        mv_status st = find_volume(c, only_id, &v);
        if (st) return st;
        if (!v->resident) return fail(c, MV_ERR_NOT_RESIDENT, "volume is swapped out");
    }
    mv_status st = begin_call(c, s, only_id);
    if (st) return st;
    const FrameParams P = make_params(c, K, T);
    int slot0 = 0, nvol = (int)c->table.size();
    if (only_id >= 0) {
        slot0 = table_slot(c, only_id);
        nvol = 1;
    }
    const VolDev *tab = c->d_table + slot0;
    VolFrame *vf = c->d_vf + slot0;
    VisList *vis = (only_id >= 0 || nvol == 0) ? nullptr : c->d_vis;
    if (nvol > 0)
        MV_CUDA(c, counted_launch(c, MV_KERNEL_SETUP, s, [&] {
            return launch_frame_setup(tab, nvol, P, vf, nullptr, s, vis); }));
    MV_CUDA(c, counted_launch(c, MV_KERNEL_RAYCAST, s, [&] {
        return launch_raycast(tab, vf, nvol, P, depth, normal, rgba, vertex, vol_id, merge ? 1 : 0,
                              c->d_stats, c->ray_tile, s, vis); }));
    return end_call(c, s);
}

mv_status mv_raycast(mv_ctx *c, const mv_intrinsics *K, const double T[16], float *depth,
                     float *normal, uint8_t *rgba, float *vertex, int32_t *vol_id, void *stream)
{
    return raycast_impl(c, -1, 1, K, T, depth, normal, rgba, vertex, vol_id, stream);
}

mv_status mv_raycast_batch(mv_ctx *c, const mv_intrinsics *K, const double *T, int32_t n_views, float *depth,
                           float *normal, uint8_t *rgba, float *vertex, int32_t *vol_id, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!T || n_views < 1 || n_views > 65535) return fail(c, MV_ERR_ARG, "bad view count");
    for (int k = 0; k < n_views; ++k)
        if (!valid_frame(K, T + 16 * (size_t)k)) return fail(c, MV_ERR_ARG, "bad view arguments");
    if (!aligned_to({depth, normal, rgba, vertex, vol_id}, 4))
        return fail(c, MV_ERR_ARG, "maps must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    mv_status st = begin_call(c, s);
    if (st) return st;
    if (n_views > c->batch_cap) {
        // earlier calls may still read the old buffers
        MV_CUDA(c, cudaStreamSynchronize(s));
        cudaFree(c->d_pb);
        cudaFree(c->d_vfb);
        cudaFree(c->d_visb);
        c->d_pb = nullptr;
        c->d_vfb = nullptr;
        c->d_visb = nullptr;
        c->batch_cap = 0;
        MV_CUDA(c, cudaMalloc((void **)&c->d_pb, sizeof(FrameParams) * n_views));
        MV_CUDA(c, cudaMalloc((void **)&c->d_vfb, sizeof(VolFrame) * (size_t)kMaxVolumes * n_views));
        MV_CUDA(c, cudaMalloc((void **)&c->d_visb, sizeof(VisList) * n_views));
        c->batch_cap = n_views;
    }
    const int nvol = (int)c->table.size();
    c->h_pb.resize(n_views);
    for (int k = 0; k < n_views; ++k) c->h_pb[k] = make_params(c, K, T + 16 * (size_t)k);
    st = upload_small(c, c->d_pb, c->h_pb.data(), sizeof(FrameParams) * n_views, s);
    if (st) return st;
    if (nvol > 0)
        for (int k = 0; k < n_views; ++k)
            MV_CUDA(c, counted_launch(c, MV_KERNEL_SETUP, s, [&] {
                return launch_frame_setup(c->d_table, nvol, c->h_pb[k], c->d_vfb + (size_t)k * nvol, nullptr, s,
                                          c->d_visb + k); }));
    MV_CUDA(c, counted_launch(c, MV_KERNEL_RAYCAST, s, [&] {
        return launch_raycast_batch(c->d_table, c->d_vfb, nvol, c->d_pb, n_views, K->width, K->height, depth,
                                    normal, rgba, vertex, vol_id, c->d_stats, c->ray_tile, s,
                                    nvol > 0 ? c->d_visb : nullptr); }));
    return end_call(c, s);
}

mv_status mv_raycast_volume(mv_ctx *c, int32_t id, int32_t first, const mv_intrinsics *K,
                            const double T[16], float *depth, float *normal, uint8_t *rgba,
                            float *vertex, int32_t *vol_id, void *stream)
{
    if (id < 0) return fail(c, MV_ERR_NOT_FOUND, "negative id");
    return raycast_impl(c, id, first, K, T, depth, normal, rgba, vertex, vol_id, stream);
}

mv_status mv_frame(mv_ctx *c, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                   const double T[16], float *depth_out, float *normal, uint8_t *rgba, float *vertex,
                   int32_t *vol_id, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!depth || !valid_frame(K, T)) return fail(c, MV_ERR_ARG, "bad frame arguments");
    if (!aligned_to({depth, depth_out, normal, rgba, vertex, vol_id}, 4))
        return fail(c, MV_ERR_ARG, "depth and maps must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    mv_status st = begin_call(c, s);
    if (st) return st;
    st = ensure_pyramid(c, K);
    if (st) return st;
    const FrameParams P = make_params(c, K, T);
    const int nvol = (int)c->table.size();
    if (nvol == 0) {  // nothing to integrate: the maps are all misses
        MV_CUDA(c, counted_launch(c, MV_KERNEL_RAYCAST, s, [&] {
            return launch_raycast(c->d_table, c->d_vf, 0, P, depth_out, normal, rgba, vertex, vol_id, 0,
                                  c->d_stats, c->ray_tile, s, nullptr); }));
        return end_call(c, s);
    }
    const long long total = c->table.back().brick_base + c->table.back().nbricks;
    const bool two_level = two_level_list(c);
    auto &fg = c->fg;
    const bool rebuild = !fg.exec || fg.table_version != c->table_version || fg.width != K->width ||
                         fg.height != K->height || fg.grid_int != c->grid_integrate ||
                         fg.tile != c->ray_tile || fg.two_level != two_level;
    if (rebuild) {
        if (fg.exec) cudaGraphExecDestroy(fg.exec);
        if (fg.g) cudaGraphDestroy(fg.g);
        fg.exec = nullptr;
        fg.g = nullptr;
        MV_CUDA(c, cudaGraphCreate(&fg.g, 0));
    }
    cudaGraphExec_t upd = rebuild ? nullptr : fg.exec;
    MV_CUDA(c, graph_integrate(fg.g, upd, fg.nodes, nullptr, c->d_table, nvol, c->d_vf, P, total, c->total_sup,
                               two_level ? c->d_slist : nullptr, c->d_list, c->d_counter, depth, rgb,
                               c->d_stats, c->grid_integrate,
                               c->num_sms, c->d_vis, c->d_list + c->list_cap, ++c->integrations, c->d_pyr));
    MV_CUDA(c, graph_raycast(fg.g, upd, &fg.nodes[6], fg.nodes[5], c->d_table, nvol, c->d_vf, P,
                             depth_out, normal, rgba, vertex, vol_id, c->d_stats, c->ray_tile, c->d_vis));
    if (rebuild) {
        MV_CUDA(c, cudaGraphInstantiate(&fg.exec, fg.g, 0));
        fg.table_version = c->table_version;
        fg.width = K->width;
        fg.height = K->height;
        fg.grid_int = c->grid_integrate;
        fg.tile = c->ray_tile;
        fg.two_level = two_level;
    }
    MV_CUDA(c, counted_launch(c, MV_KERNEL_FRAME_GRAPH, s, [&] { return cudaGraphLaunch(fg.exec, s); }));
    const int kinds[6] = {MV_KERNEL_SETUP, MV_KERNEL_DEPTH_MAX, MV_KERNEL_BRICK_LIST, MV_KERNEL_INTEGRATE,
                          MV_KERNEL_CELL_FLAGS, MV_KERNEL_RAYCAST};
    for (int k : kinds) c->launches[k] += 1;
    if (two_level) c->launches[MV_KERNEL_BRICK_LIST] += 1;
    return end_call(c, s);
}

mv_status mv_frame_host(mv_ctx *c, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                        const double T[16], float *depth_out, float *normal, uint8_t *rgba, float *vertex,
                        int32_t *vol_id, uint64_t *ticket)
{
    if (!c) return MV_ERR_ARG;
    if (!depth || !ticket || !valid_frame(K, T)) return fail(c, MV_ERR_ARG, "bad frame arguments");
    cudaSetDevice(c->device);
    MV_CUDA(c, ensure_host_pipe(c, K->width, K->height));
    auto &hp = c->hp;
    const int b = (int)(hp.next & 1u);
    const size_t n = (size_t)K->width * (size_t)K->height;
    // upload: the set's inputs are free once the frame that used them last has run
    if (hp.used[b]) MV_CUDA(c, cudaStreamWaitEvent(hp.up, hp.computed[b], 0));
    MV_CUDA(c, cudaMemcpyAsync(hp.depth[b], depth, n * 4, cudaMemcpyHostToDevice, hp.up));
    if (rgb) MV_CUDA(c, cudaMemcpyAsync(hp.rgb[b], rgb, n * 3, cudaMemcpyHostToDevice, hp.up));
    MV_CUDA(c, cudaEventRecord(hp.uploaded[b], hp.up));
    // run: after this frame's upload and the download of the set's last maps
    MV_CUDA(c, cudaStreamWaitEvent(hp.run, hp.uploaded[b], 0));
    if (hp.used[b]) MV_CUDA(c, cudaStreamWaitEvent(hp.run, hp.downloaded[b], 0));
    mv_status st = mv_frame(c, hp.depth[b], rgb ? hp.rgb[b] : nullptr, K, T, hp.dout[b],
                            normal ? hp.normal[b] : nullptr, rgba ? hp.rgba[b] : nullptr,
                            vertex ? hp.vertex[b] : nullptr, hp.vid[b], hp.run);
    if (st) return st;
    MV_CUDA(c, cudaEventRecord(hp.computed[b], hp.run));
    // download of the requested maps
    MV_CUDA(c, cudaStreamWaitEvent(hp.down, hp.computed[b], 0));
    if (depth_out) MV_CUDA(c, cudaMemcpyAsync(depth_out, hp.dout[b], n * 4, cudaMemcpyDeviceToHost, hp.down));
    if (normal) MV_CUDA(c, cudaMemcpyAsync(normal, hp.normal[b], n * 12, cudaMemcpyDeviceToHost, hp.down));
    if (rgba) MV_CUDA(c, cudaMemcpyAsync(rgba, hp.rgba[b], n * 4, cudaMemcpyDeviceToHost, hp.down));
    if (vertex) MV_CUDA(c, cudaMemcpyAsync(vertex, hp.vertex[b], n * 12, cudaMemcpyDeviceToHost, hp.down));
    if (vol_id) MV_CUDA(c, cudaMemcpyAsync(vol_id, hp.vid[b], n * 4, cudaMemcpyDeviceToHost, hp.down));
    MV_CUDA(c, cudaEventRecord(hp.downloaded[b], hp.down));
    hp.used[b] = true;
    *ticket = hp.next++;
    return MV_OK;
}

mv_status mv_frame_host_wait(mv_ctx *c, uint64_t ticket)
{
    if (!c) return MV_ERR_ARG;
    auto &hp = c->hp;
    if (ticket >= hp.next) return fail(c, MV_ERR_ARG, "no such frame");
    cudaSetDevice(c->device);
    // the set's download event is that of the latest frame on the set, which
    // finishes after every earlier frame's download (one download stream)
    MV_CUDA(c, cudaEventSynchronize(hp.downloaded[ticket & 1u]));
    return MV_OK;
}

mv_status mv_frame_streamed(mv_ctx *c, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                            const double T[16], float *depth_out, float *normal, uint8_t *rgba,
                            float *vertex, int32_t *vol_id, int32_t n_slots, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!depth || !valid_frame(K, T)) return fail(c, MV_ERR_ARG, "bad frame arguments");
    if (!depth_out || !vol_id) return fail(c, MV_ERR_ARG, "depth_out and vol_id are required");
    if (n_slots < 1 || n_slots > kMaxStreamSlots) return fail(c, MV_ERR_ARG, "n_slots out of range");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    // 1. resident volumes: batched integration, then the raycast that
    //    initialises the maps
    mv_status st = integrate_impl(c, -1, depth, rgb, K, T, stream);
    if (st) return st;
    st = raycast_impl(c, -1, 1, K, T, depth_out, normal, rgba, vertex, vol_id, stream);
    if (st) return st;
    std::vector<Volume *> streamed;
    size_t fw = 0, col = 0, fl = 0;
    long long bricks = 0;
    for (auto &kv : c->vols) {
        Volume *v = kv.second;
        if (v->resident) continue;
        streamed.push_back(v);
        fw = std::max(fw, v->fw_bytes);
        col = std::max(col, v->rgba_bytes);
        fl = std::max(fl, v->flag_bytes);
        bricks = std::max(bricks, v->nbricks);
    }
    if (streamed.empty()) return MV_OK;
    st = begin_call(c, s);
    if (st) return st;
    st = ensure_slots(c, n_slots, fw, col, fl, bricks, s);
    if (st) return st;
    auto &ss = c->ss;
    const int n = ss.n < n_slots ? ss.n : n_slots;
    const FrameParams P = make_params(c, K, T);
    // the copies start after everything queued on the caller's stream so far
    MV_CUDA(c, cudaEventRecord(c->last_event, s));
    MV_CUDA(c, cudaStreamWaitEvent(ss.h2d, c->last_event, 0));
    // 2. every swapped-out volume passes through a slot: its flags and the
    //    bricks the frame can read are uploaded (the bricks by a gather kernel
    //    reading the mapped host copy), it is integrated and raycast into the
    //    maps (nearest hit wins, as between resident volumes), and its flags
    //    and the bricks the integration changed are written back; slot j is
    //    reused once its previous volume is written back
    for (size_t i = 0; i < streamed.size(); ++i) {
        Volume *v = streamed[i];
        const int j = (int)(i % (size_t)n);
        unsigned *cnt = ss.counter + 4 * j;
        uint2 *list = ss.list[j];
        void *hfw = nullptr, *hcol = nullptr;
        MV_CUDA(c, cudaHostGetDevicePointer(&hfw, v->h_fw, 0));
        MV_CUDA(c, cudaHostGetDevicePointer(&hcol, v->h_rgba, 0));
        Volume staged = *v;
        staged.d_fw = ss.fw[j];
        staged.d_rgba = ss.rgba[j];
        staged.d_flag = ss.flag[j];
        VolDev d = make_voldev(staged);
        d.brick_base = 0;
        VolDev *dv = ss.d_vol + j;
        VolFrame *vf = ss.d_vf + j;

        cudaStream_t up = ss.h2d;
        if (ss.freed_rec[j]) MV_CUDA(c, cudaStreamWaitEvent(up, ss.freed[j], 0));
        if (v->ready_pending) MV_CUDA(c, cudaStreamWaitEvent(up, v->ready, 0));
        MV_CUDA(c, cudaMemcpyAsync(ss.flag[j], v->h_flag, v->flag_bytes, cudaMemcpyHostToDevice, up));
        put_voldev_kernel<<<1, 32, 0, up>>>(d, dv);
        MV_CUDA(c, cudaGetLastError());
        MV_CUDA(c, counted_launch(c, MV_KERNEL_SETUP, up, [&] {
            return launch_frame_setup(dv, 1, P, vf, cnt, up, nullptr); }));
        MV_CUDA(c, counted_launch(c, MV_KERNEL_STREAM, up, [&] {
            return launch_stream_gather(d, vf, P, hfw, hcol, &c->d_stats->stream_up, c->num_sms, up); }));
        MV_CUDA(c, cudaEventRecord(ss.loaded[j], up));

        MV_CUDA(c, cudaStreamWaitEvent(s, ss.loaded[j], 0));
        MV_CUDA(c, counted_launch(c, MV_KERNEL_DEPTH_MAX, s, [&] {
            return launch_depth_max(depth, P, cnt + 1, c->num_sms, s, c->d_pyr); }));
        MV_CUDA(c, counted_launch(c, MV_KERNEL_BRICK_LIST, s, [&] {
            return launch_brick_list(dv, 1, vf, P, 0, v->nbricks, list, cnt, c->num_sms, s, nullptr, cnt + 1,
                                     c->d_pyr, nullptr, 0); }));
        MV_CUDA(c, counted_launch(c, MV_KERNEL_INTEGRATE, s, [&] {
            return launch_integrate(dv, vf, list, cnt, P, depth, rgb, c->d_stats, c->grid_integrate, s,
                                    nullptr, nullptr, 0u); }));
        MV_CUDA(c, counted_launch(c, MV_KERNEL_CELL_FLAGS, s, [&] {
            return launch_cell_flags(dv, list, cnt, c->num_sms, s); }));
        MV_CUDA(c, counted_launch(c, MV_KERNEL_RAYCAST, s, [&] {
            return launch_raycast(dv, vf, 1, P, depth_out, normal, rgba, vertex, vol_id, 1, c->d_stats,
                                  c->ray_tile, s, nullptr); }));
        MV_CUDA(c, cudaEventRecord(ss.done[j], s));

        cudaStream_t down = ss.d2h;
        MV_CUDA(c, cudaStreamWaitEvent(down, ss.done[j], 0));
        MV_CUDA(c, counted_launch(c, MV_KERNEL_STREAM, down, [&] {
            return launch_stream_scatter(d, list, cnt, hfw, hcol, &c->d_stats->stream_down, c->num_sms, down); }));
        MV_CUDA(c, cudaMemcpyAsync(v->h_flag, ss.flag[j], v->flag_bytes, cudaMemcpyDeviceToHost, down));
        MV_CUDA(c, cudaEventRecord(ss.freed[j], down));
        ss.freed_rec[j] = true;
        // later readers of the host copy (swap-in, read, write) wait for it
        MV_CUDA(c, cudaEventRecord(v->ready, down));
        v->ready_pending = true;
    }
    // the caller's stream continues once every download has finished
    for (int j = 0; j < n; ++j)
        if (ss.freed_rec[j]) MV_CUDA(c, cudaStreamWaitEvent(s, ss.freed[j], 0));
    return end_call(c, s);
}

static float time_ms(cudaStream_t s, cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

mv_status mv_autotune(mv_ctx *c, const float *depth, const uint8_t *rgb, const mv_intrinsics *K,
                      const double T[16], mv_tuning *out, void *stream)
{
    if (!c || !out) return MV_ERR_ARG;
    if (!depth || !valid_frame(K, T)) return fail(c, MV_ERR_ARG, "bad frame arguments");
    if (!aligned_to({depth}, 4)) return fail(c, MV_ERR_ARG, "depth must be 4-byte aligned");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    mv_status st = begin_call(c, s);
    if (st) return st;
    st = ensure_pyramid(c, K);
    if (st) return st;
    std::memset(out, 0, sizeof(*out));
    const FrameParams P = make_params(c, K, T);
    const int nvol = (int)c->table.size();
    cudaEvent_t a, b;
    MV_CUDA(c, cudaEventCreate(&a));
    MV_CUDA(c, cudaEventCreate(&b));
    const size_t npx = (size_t)K->width * K->height;
    char *maps = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&maps, npx * 36, s);
    // raycast tile shapes on the resident volumes (the raycast changes no state);
    // median of 5 timed launches per shape, the current shape kept unless
    // another is faster by more than 3 %
    float best = 3.0e38f, t_cur = 3.0e38f;
    int best_tile = c->ray_tile, cand_tile = c->ray_tile;
    for (int tile = 0; tile < 4 && e == cudaSuccess; ++tile) {
        float t[5];
        int nt = 0;
        for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
            e = launch_frame_setup(c->d_table, nvol, P, c->d_vf, nullptr, s, c->d_vis);
            if (e == cudaSuccess) e = cudaEventRecord(a, s);
            if (e == cudaSuccess)
                e = launch_raycast(c->d_table, c->d_vf, nvol, P, (float *)maps, (float *)(maps + 4 * npx),
                                   (uint8_t *)(maps + 16 * npx), (float *)(maps + 20 * npx),
                                   (int *)(maps + 32 * npx), 0, nullptr, tile, s, c->d_vis);
            if (e == cudaSuccess) e = cudaEventRecord(b, s);
            if (e == cudaSuccess && rep > 0) t[nt++] = time_ms(s, a, b);
        }
        if (e != cudaSuccess) break;
        std::sort(t, t + nt);
        const float med = t[nt / 2];
        out->raycast_ms[tile] = med;
        if (tile == c->ray_tile) t_cur = med;
        if (med < best) { best = med; cand_tile = tile; }
    }
    if (best < 0.97f * t_cur) best_tile = cand_tile;
    if (maps) cudaFreeAsync(maps, s);
    // persistent-grid sizes of the integration, on scratch storage shaped like
    // the largest volume in view (the map itself is not touched)
    int best_ctas = c->ctas_per_sm;
    int big = -1;
    if (e == cudaSuccess && nvol > 0) {
        int nvis = 0;
        e = cudaMemcpyAsync(&nvis, &c->d_vis->count, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        nvis = std::min(std::max(nvis, 0), nvol);
        std::vector<int> vis_slots((size_t)nvis);
        if (e == cudaSuccess && nvis > 0) {
            e = cudaMemcpyAsync(vis_slots.data(), c->d_vis->slot, sizeof(int) * (size_t)nvis,
                                cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        for (int k = 0; k < nvis && e == cudaSuccess; ++k) {
            const int i = vis_slots[(size_t)k];
            if (i >= 0 && i < nvol && (big < 0 || c->table[i].nbricks > c->table[big].nbricks)) big = i;
        }
    }
    if (e == cudaSuccess && big >= 0) {
        VolDev sv = c->table[big];
        const Volume *vol = c->vols.at(sv.id);
        void *sfw = nullptr, *srgba = nullptr, *sflag = nullptr;
        VolDev *stab = nullptr;
        VolFrame *svf = nullptr;
        uint2 *slist = nullptr;
        unsigned *scount = nullptr;
        e = cudaMallocAsync(&sfw, vol->fw_bytes, s);
        if (e == cudaSuccess) e = cudaMallocAsync(&srgba, vol->rgba_bytes, s);
        if (e == cudaSuccess) e = cudaMallocAsync(&sflag, vol->flag_bytes, s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&stab, sizeof(VolDev), s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&svf, sizeof(VolFrame), s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&slist, sizeof(uint2) * sv.nbricks, s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&scount, sizeof(unsigned) * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sfw, 0, vol->fw_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(srgba, 0, vol->rgba_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sflag, kFlagsNew, (size_t)sv.nbricks, s);
        sv.fw = sfw;
        sv.rgba = (uint32_t *)srgba;
        sv.bflag = (uint8_t *)sflag;
        sv.cflag = nullptr;
        sv.surf = nullptr;
        sv.sup = nullptr;
        sv.vmask = nullptr;
        sv.cmask = nullptr;
        sv.stamp = nullptr;
        sv.brick_base = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(stab, &sv, sizeof(VolDev), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // sv is a stack value
        const int maxc = integrate_max_ctas_per_sm();
        const int cands[5] = {2, 4, 6, 8, 10};
        // median of 5 timed launches per size; the default size is kept unless
        // another is faster by more than 3 %
        float t_default = 3.0e38f, ibest = 3.0e38f;
        int cand_best = best_ctas;
        for (int ci = 0; ci < 5 && e == cudaSuccess; ++ci) {
            const int ctas = cands[ci];
            if (ctas > maxc) break;
            float t[5];
            int nt = 0;
            for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
                e = launch_frame_setup(stab, 1, P, svf, scount, s, nullptr);
                if (e == cudaSuccess) e = launch_depth_max(depth, P, scount + 1, c->num_sms, s, c->d_pyr);
                if (e == cudaSuccess)
                    e = launch_brick_list(stab, 1, svf, P, 0, sv.nbricks, slist, scount, c->num_sms, s,
                                          nullptr, scount + 1, c->d_pyr, nullptr, 0);
                if (e == cudaSuccess) e = cudaEventRecord(a, s);
                if (e == cudaSuccess)
                    e = launch_integrate(stab, svf, slist, scount, P, depth, rgb, nullptr,
                                         c->num_sms * ctas, s, nullptr, nullptr, 0u);
                if (e == cudaSuccess) e = cudaEventRecord(b, s);
                if (e == cudaSuccess && rep > 0) t[nt++] = time_ms(s, a, b);
            }
            if (e != cudaSuccess) break;
            std::sort(t, t + nt);
            const float med = t[nt / 2];
            out->integrate_ms[ci] = med;
            if (ctas == best_ctas) t_default = med;
            if (med < ibest) { ibest = med; cand_best = ctas; }
        }
        if (ibest < 0.97f * t_default) best_ctas = cand_best;
        for (void *p : {sfw, srgba, sflag, (void *)stab, (void *)svf, (void *)slist, (void *)scount})
            if (p) cudaFreeAsync(p, s);
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(c, e, "autotune");
    }
    c->ray_tile = best_tile;
    c->ctas_per_sm = best_ctas;
    c->grid_integrate = c->num_sms * best_ctas;
    out->raycast_tile = best_tile;
    out->integrate_ctas_per_sm = best_ctas;
    out->work_list_levels = c->list_levels;
    return end_call(c, s);
}

mv_status mv_set_tuning(mv_ctx *c, const mv_tuning *t)
{
    if (!c || !t) return MV_ERR_ARG;
    if (t->raycast_tile < 0 || t->raycast_tile > 3 || t->integrate_ctas_per_sm < 1 ||
        t->integrate_ctas_per_sm > integrate_max_ctas_per_sm() || t->work_list_levels < 0 ||
        t->work_list_levels > 2)
        return fail(c, MV_ERR_ARG, "bad tuning values");
    c->list_levels = t->work_list_levels;
    c->ray_tile = t->raycast_tile;
    c->ctas_per_sm = t->integrate_ctas_per_sm;
    c->grid_integrate = c->num_sms * t->integrate_ctas_per_sm;
    return MV_OK;
}

mv_status mv_get_tuning(mv_ctx *c, mv_tuning *t)
{
    if (!c || !t) return MV_ERR_ARG;
    std::memset(t, 0, sizeof(*t));
    t->raycast_tile = c->ray_tile;
    t->integrate_ctas_per_sm = c->ctas_per_sm;
    t->work_list_levels = c->list_levels;
    return MV_OK;
}

// The L1 loss of pose refinement formed on the device (mv_raycast_backward_l1).
struct L1Loss {
    const uint8_t *rgba;
    const float *ref_depth;
    const uint8_t *ref_rgba;
    float colour_weight;
    float *loss;
};

static mv_status raycast_backward_impl(mv_ctx *c, const mv_intrinsics *K, const double *T, int32_t n_poses,
                                       const float *depth, const int32_t *vol_id, const float *grad_depth,
                                       const float *grad_rgb, float *grad_pose, const mv_grad_target *targets,
                                       int32_t n_targets, void *stream, const L1Loss *l1)
{
    if (!c) return MV_ERR_ARG;
    if (n_poses < 1 || n_poses > 65535 || !depth || !vol_id || !grad_pose || (n_targets > 0 && !targets) ||
        n_targets < 0)
        return fail(c, MV_ERR_ARG, "bad backward arguments");
    if (!aligned_to({depth, vol_id, grad_depth, grad_rgb, grad_pose}, 4))
        return fail(c, MV_ERR_ARG, "backward buffers must be 4-byte aligned");
    for (int i = 0; i < n_targets; ++i)
        if (!aligned_to({targets[i].grad_tsdf}, 4)) return fail(c, MV_ERR_ARG, "gradient buffers must be 4-byte aligned");
    for (int i = 0; i < n_poses; ++i)
        if (!valid_frame(K, T + 16 * i)) return fail(c, MV_ERR_ARG, "bad view arguments");
    for (int i = 0; i < n_targets; ++i) {
        Volume *v;
        mv_status st = find_volume(c, targets[i].id, &v);
        if (st) return st;
        if (!targets[i].grad_tsdf) return fail(c, MV_ERR_ARG, "null gradient buffer");
        if (!v->resident) return fail(c, MV_ERR_NOT_RESIDENT, "gradient target is swapped out");
    }
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    mv_status st = begin_call(c, s);
    if (st) return st;
    // per pose its rotation and translation in float, and per pose and table
    // slot the camera position in that volume's voxel coordinates (in double,
    // rounded once): the kernel then needs no FP64 arithmetic
    const size_t nslot = c->table.size();
    const size_t nf = 12 * (size_t)n_poses + 3 * (size_t)n_poses * nslot;
    if (nf > c->poses_cap) {
        if (c->d_poses) MV_CUDA(c, cudaFreeAsync(c->d_poses, s));
        c->d_poses = nullptr;
        c->poses_cap = 0;
        MV_CUDA(c, cudaMallocAsync((void **)&c->d_poses, sizeof(float) * nf, s));
        c->poses_cap = nf;
    }
    c->h_pose_f.resize(nf);
    for (int i = 0; i < n_poses; ++i) {
        const double *Ti = T + 16 * (size_t)i;
        float *pf = c->h_pose_f.data() + 12 * (size_t)i;
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) pf[3 * a + b] = (float)Ti[4 * a + b];
            pf[9 + a] = (float)Ti[4 * a + 3];
        }
        float *cf = c->h_pose_f.data() + 12 * (size_t)n_poses + 3 * (size_t)i * nslot;
        for (size_t k = 0; k < nslot; ++k)
            for (int a = 0; a < 3; ++a)
                cf[3 * k + a] = (float)(Ti[4 * a + 3] / (double)c->table[k].s - (double)c->table[k].h[a]);
    }
    st = upload_small(c, c->d_poses, c->h_pose_f.data(), sizeof(float) * nf, s);
    if (st) return st;
    std::vector<float *> ptrs(c->table.size() > 0 ? c->table.size() : 1, nullptr);
    for (int i = 0; i < n_targets; ++i) {
        const int slot = table_slot(c, targets[i].id);
        if (slot >= 0) ptrs[slot] = targets[i].grad_tsdf;
    }
    if (!c->table.empty()) {
        st = upload_small(c, c->d_grad_ptrs, ptrs.data(), sizeof(float *) * c->table.size(), s);
        if (st) return st;
    }
    MV_CUDA(c, cudaMemsetAsync(grad_pose, 0, sizeof(float) * 6 * n_poses, s));
    BackwardArgs A;
    A.vols = c->d_table;
    A.nvol = (int)c->table.size();
    A.grad_tsdf = c->d_grad_ptrs;
    A.pose_f = c->d_poses;
    A.cam_f = c->d_poses + 12 * (size_t)n_poses;
    A.n_poses = n_poses;
    A.fx = K->fx; A.fy = K->fy; A.cx = K->cx; A.cy = K->cy;
    A.width = K->width; A.height = K->height;
    A.depth = depth;
    A.vol_id = vol_id;
    A.grad_depth = grad_depth;
    A.grad_rgb = grad_rgb;
    A.grad_pose = grad_pose;
    const size_t need = backward_ctas_per_pose(K->width, K->height) * 6 * (size_t)n_poses;
    if (need > c->bw_partial_cap) {
        if (c->d_bw_partial) MV_CUDA(c, cudaFreeAsync(c->d_bw_partial, s));
        c->d_bw_partial = nullptr;
        c->bw_partial_cap = 0;
        MV_CUDA(c, cudaMallocAsync((void **)&c->d_bw_partial, sizeof(float) * need, s));
        c->bw_partial_cap = need;
    }
    A.partial = c->d_bw_partial;
    A.rgba = nullptr;
    A.ref_depth = nullptr;
    A.ref_rgba = nullptr;
    A.colour_weight = 0.f;
    A.l1_count = nullptr;
    if (l1) {
        if (!c->d_l1) {
            MV_CUDA(c, cudaMallocAsync((void **)&c->d_l1, kL1ScratchBytes, s));
            MV_CUDA(c, cudaMemsetAsync(c->d_l1, 0, kL1ScratchBytes, s));
        }
        const long long npx = (long long)n_poses * K->width * K->height;
        MV_CUDA(c, counted_launch(c, MV_KERNEL_BACKWARD, s, [&] {
            return launch_l1_stats(depth, l1->ref_depth, l1->rgba, l1->ref_rgba, npx, l1->colour_weight, c->d_l1,
                                   l1->loss, s); }));
        A.rgba = l1->rgba;
        A.ref_depth = l1->ref_depth;
        A.ref_rgba = l1->ref_rgba;
        A.colour_weight = l1->colour_weight;
        A.l1_count = c->d_l1 + 1;
    }
    if (A.nvol > 0)
        MV_CUDA(c, counted_launch(c, MV_KERNEL_BACKWARD, s, [&] { return launch_raycast_backward(A, s); }));
    return end_call(c, s);
}

mv_status mv_raycast_backward(mv_ctx *c, const mv_intrinsics *K, const double *T, int32_t n_poses,
                              const float *depth, const int32_t *vol_id, const float *grad_depth,
                              const float *grad_rgb, float *grad_pose, const mv_grad_target *targets,
                              int32_t n_targets, void *stream)
{
    return raycast_backward_impl(c, K, T, n_poses, depth, vol_id, grad_depth, grad_rgb, grad_pose, targets,
                                 n_targets, stream, nullptr);
}

mv_status mv_raycast_backward_l1(mv_ctx *c, const mv_intrinsics *K, const double *T, int32_t n_poses,
                                 const float *depth, const uint8_t *rgba, const int32_t *vol_id,
                                 const float *ref_depth, const uint8_t *ref_rgba, float colour_weight,
                                 float *grad_pose, float *loss, void *stream)
{
    if (!c) return MV_ERR_ARG;
    if (!rgba || !ref_depth || !ref_rgba || !loss || !std::isfinite(colour_weight))
        return fail(c, MV_ERR_ARG, "bad L1 loss arguments");
    // the kernels read a pixel's colour as one 4-byte word and its depths as floats
    if ((reinterpret_cast<uintptr_t>(rgba) | reinterpret_cast<uintptr_t>(ref_rgba) |
         reinterpret_cast<uintptr_t>(depth) | reinterpret_cast<uintptr_t>(ref_depth) |
         reinterpret_cast<uintptr_t>(loss)) & 3u)
        return fail(c, MV_ERR_ARG, "L1 loss buffers must be 4-byte aligned");
    const L1Loss l1{rgba, ref_depth, ref_rgba, colour_weight, loss};
    return raycast_backward_impl(c, K, T, n_poses, depth, vol_id, nullptr, nullptr, grad_pose, nullptr, 0, stream,
                                 &l1);
}

mv_status mv_swap_out(mv_ctx *c, int32_t id, void *stream)
{
    if (!c) return MV_ERR_ARG;
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    if (!v->resident) return MV_OK;
    cudaSetDevice(c->device);
    if (!v->h_fw) {
        v->h_fw = c->pool->take(v->fw_bytes);
        v->h_rgba = (uint32_t *)c->pool->take(v->rgba_bytes);
        v->h_flag = (uint8_t *)c->pool->take(v->flag_bytes);
        if (!v->h_fw || !v->h_rgba || !v->h_flag) {
            free_host(c, v);
            return fail(c, MV_ERR_OOM, "pinned host allocation failed");
        }
    }
    cudaStream_t s = c->swap_stream;
    // after all earlier work of the context and of the caller's stream
    if (c->last_recorded) MV_CUDA(c, cudaStreamWaitEvent(s, c->last_event, 0));
    MV_CUDA(c, cudaEventRecord(c->last_event, (cudaStream_t)stream));
    MV_CUDA(c, cudaStreamWaitEvent(s, c->last_event, 0));
    if (v->ready_pending) MV_CUDA(c, cudaStreamWaitEvent(s, v->ready, 0));
    MV_CUDA(c, cudaMemcpyAsync(v->h_fw, v->d_fw, v->fw_bytes, cudaMemcpyDeviceToHost, s));
    MV_CUDA(c, cudaMemcpyAsync(v->h_rgba, v->d_rgba, v->rgba_bytes, cudaMemcpyDeviceToHost, s));
    MV_CUDA(c, cudaMemcpyAsync(v->h_flag, v->d_flag, v->flag_bytes, cudaMemcpyDeviceToHost, s));
    MV_CUDA(c, cudaFreeAsync(v->d_fw, s));
    MV_CUDA(c, cudaFreeAsync(v->d_rgba, s));
    MV_CUDA(c, cudaFreeAsync(v->d_flag, s));
    if (v->d_mask) MV_CUDA(c, cudaFreeAsync(v->d_mask, s));
    MV_CUDA(c, cudaEventRecord(v->ready, s));
    v->ready_pending = true;
    v->d_fw = nullptr;
    v->d_rgba = nullptr;
    v->d_flag = nullptr;
    v->d_mask = nullptr;
    v->resident = false;
    c->table_dirty = true;
    return MV_OK;
}

mv_status mv_swap_in(mv_ctx *c, int32_t id, void *stream)
{
    if (!c) return MV_ERR_ARG;
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    if (v->resident) return MV_OK;
    cudaSetDevice(c->device);
    cudaStream_t s = c->swap_stream;
    (void)stream;
    // a download into the host copy (swap-out or streamed frame) may still run
    if (v->ready_pending) MV_CUDA(c, cudaStreamWaitEvent(s, v->ready, 0));
    void *fw = nullptr, *rgba = nullptr, *flag = nullptr, *mask = nullptr;
    cudaError_t e = cudaMallocAsync(&fw, v->fw_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&rgba, v->rgba_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&flag, v->flag_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&mask, mask_alloc_bytes(v->nbricks), s);
    if (e != cudaSuccess) {
        if (fw) cudaFreeAsync(fw, s);
        if (rgba) cudaFreeAsync(rgba, s);
        if (flag) cudaFreeAsync(flag, s);
        if (mask) cudaFreeAsync(mask, s);
        cudaGetLastError();
        return cuda_fail(c, e, "allocating GPU memory for swap-in");
    }
    MV_CUDA(c, cudaMemcpyAsync(fw, v->h_fw, v->fw_bytes, cudaMemcpyHostToDevice, s));
    MV_CUDA(c, cudaMemcpyAsync(rgba, v->h_rgba, v->rgba_bytes, cudaMemcpyHostToDevice, s));
    MV_CUDA(c, cudaMemcpyAsync(flag, v->h_flag, v->flag_bytes, cudaMemcpyHostToDevice, s));
    v->d_fw = fw;
    v->d_rgba = (uint32_t *)rgba;
    v->d_flag = (uint8_t *)flag;
    v->d_mask = mask;
    // the masks are rebuilt from the voxels just uploaded
    const VolDev dv = make_voldev(*v);
    MV_CUDA(c, counted_launch(c, MV_KERNEL_FLAGS, s, [&] { return launch_mask_rebuild(dv, c->num_sms, s); }));
    MV_CUDA(c, cudaEventRecord(v->ready, s));
    v->ready_pending = true;
    v->resident = true;
    c->table_dirty = true;
    return MV_OK;
}

mv_status mv_read_volume(mv_ctx *c, int32_t id, void *host_fw, uint8_t *host_rgba)
{
    if (!c || !host_fw) return fail(c, MV_ERR_ARG, "null argument");
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    cudaSetDevice(c->device);
    st = wait_all(c);
    if (st) return st;
    if (v->ready_pending) MV_CUDA(c, cudaEventSynchronize(v->ready));
    std::vector<uint8_t> fw, col;
    const void *src_fw = v->h_fw;
    const void *src_col = v->h_rgba;
    if (v->resident) {
        fw.resize(v->fw_bytes);
        MV_CUDA(c, cudaMemcpy(fw.data(), v->d_fw, v->fw_bytes, cudaMemcpyDeviceToHost));
        src_fw = fw.data();
        if (host_rgba) {
            col.resize(v->rgba_bytes);
            MV_CUDA(c, cudaMemcpy(col.data(), v->d_rgba, v->rgba_bytes, cudaMemcpyDeviceToHost));
            src_col = col.data();
        }
    }
    if (v->desc.fmt == MV_TSDF_F32)
        bricks_to_linear(*v, (const uint64_t *)src_fw, (uint64_t *)host_fw);
    else
        bricks_to_linear(*v, (const uint32_t *)src_fw, (uint32_t *)host_fw);
    if (host_rgba) bricks_to_linear(*v, (const uint32_t *)src_col, (uint32_t *)host_rgba);
    return MV_OK;
}

mv_status mv_read_box(mv_ctx *c, int32_t id, const int32_t lo[3], const int32_t n[3], void *host_fw,
                      uint8_t *host_rgba)
{
    if (!c || !host_fw || !lo || !n) return fail(c, MV_ERR_ARG, "null argument");
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    for (int a = 0; a < 3; ++a)
        if (lo[a] < 0 || n[a] < 1 || (long long)lo[a] + n[a] > v->desc.h_r[a])
            return fail(c, MV_ERR_ARG, "box outside the volume");
    cudaSetDevice(c->device);
    st = wait_all(c);
    if (st) return st;
    if (v->ready_pending) MV_CUDA(c, cudaEventSynchronize(v->ready));
    const size_t total = (size_t)n[0] * n[1] * n[2];
    const int eb = v->desc.fmt == MV_TSDF_F32 ? 8 : 4;
    if (v->resident) {
        // gathered on the GPU into a temporary buffer, then one copy per array
        cudaStream_t s = c->swap_stream;
        void *tmp = nullptr;
        MV_CUDA(c, cudaMallocAsync(&tmp, total * 8, s));
        cudaError_t e = launch_gather_box(v->d_fw, eb, v->nb, lo, n, tmp, c->num_sms, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_fw, tmp, total * eb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && host_rgba) e = launch_gather_box(v->d_rgba, 4, v->nb, lo, n, tmp, c->num_sms, s);
        if (e == cudaSuccess && host_rgba) e = cudaMemcpyAsync(host_rgba, tmp, total * 4, cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(tmp, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        MV_CUDA(c, e);
        return MV_OK;
    }
    // swapped out: from the pinned host copy
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x) {
                const int gx = lo[0] + x, gy = lo[1] + y, gz = lo[2] + z;
                const size_t off = (size_t)((((long long)(gz >> 3) * v->nb[1] + (gy >> 3)) * v->nb[0] + (gx >> 3)) *
                                                kBrickVox +
                                            (((gz & 7) << 6) | ((gy & 7) << 3) | (gx & 7)));
                const size_t i = ((size_t)z * n[1] + y) * n[0] + x;
                if (eb == 8)
                    static_cast<uint64_t *>(host_fw)[i] = static_cast<const uint64_t *>(v->h_fw)[off];
                else
                    static_cast<uint32_t *>(host_fw)[i] = static_cast<const uint32_t *>(v->h_fw)[off];
                if (host_rgba)
                    reinterpret_cast<uint32_t *>(host_rgba)[i] = static_cast<const uint32_t *>(v->h_rgba)[off];
            }
    return MV_OK;
}

mv_status mv_write_volume(mv_ctx *c, int32_t id, const void *host_fw, const uint8_t *host_rgba)
{
    if (!c || !host_fw) return fail(c, MV_ERR_ARG, "null argument");
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    cudaSetDevice(c->device);
    st = wait_all(c);
    if (st) return st;
    if (v->ready_pending) MV_CUDA(c, cudaEventSynchronize(v->ready));
    std::vector<uint8_t> fw(v->fw_bytes, 0), col;
    if (v->desc.fmt == MV_TSDF_F32)
        linear_to_bricks(*v, (const uint64_t *)host_fw, (uint64_t *)fw.data());
    else
        linear_to_bricks(*v, (const uint32_t *)host_fw, (uint32_t *)fw.data());
    if (host_rgba) {
        col.assign(v->rgba_bytes, 0);
        linear_to_bricks(*v, (const uint32_t *)host_rgba, (uint32_t *)col.data());
    }
    if (v->resident) {
        MV_CUDA(c, cudaMemcpy(v->d_fw, fw.data(), v->fw_bytes, cudaMemcpyHostToDevice));
        if (host_rgba) MV_CUDA(c, cudaMemcpy(v->d_rgba, col.data(), v->rgba_bytes, cudaMemcpyHostToDevice));
        const VolDev d = make_voldev(*v);
        MV_CUDA(c, counted_launch(c, MV_KERNEL_FLAGS, c->swap_stream, [&] {
            return launch_brick_flags(d, c->num_sms, c->swap_stream); }));
        MV_CUDA(c, cudaStreamSynchronize(c->swap_stream));
    } else {
        std::memcpy(v->h_fw, fw.data(), v->fw_bytes);
        if (host_rgba) std::memcpy(v->h_rgba, col.data(), v->rgba_bytes);
        // exact flags on the host: voxel-brick summaries, then cell-brick flags
        const long long nb = v->nbricks;
        unsigned surf = 0;
        for (long long b = 0; b < nb; ++b) {
            bool all_free = true, all_empty = true, no_neg = true;
            for (int k = 0; k < kBrickVox; ++k) {
                float F, W;
                const size_t off = (size_t)b * kBrickVox + k;
                if (v->desc.fmt == MV_TSDF_F32) {
                    const float *q = (const float *)fw.data() + 2 * off;
                    F = q[0];
                    W = q[1];
                } else {
                    const uint32_t q = ((const uint32_t *)fw.data())[off];
                    W = (float)(q >> 16);
                    const uint16_t lo = (uint16_t)(q & 0xFFFFu);
                    if (v->desc.fmt == MV_TSDF_I16) F = (float)(int16_t)lo;
                    else F = (lo & 0x7FFFu) && !(lo & 0x8000u) ? 1.f : ((lo & 0x8000u) ? -1.f : 0.f);
                }
                const bool valid = W > 0.f;
                all_free &= valid && (F > 0.f);
                all_empty &= !valid;
                no_neg &= !valid || (F > 0.f);
            }
            v->h_flag[b] = (uint8_t)((all_free ? kFlagFree : 0) | (all_empty ? kFlagEmpty : 0) |
                                     (no_neg ? kFlagNoNeg : 0));
            surf += no_neg ? 0u : 1u;
        }
        std::memcpy(v->h_flag + flag_count_offset(nb), &surf, sizeof(surf));
        std::vector<unsigned> sup((size_t)v->nsuper, 0u);
        for (long long b = 0; b < nb; ++b) {
            const int cx = (int)(b % v->nb[0]), cy = (int)((b / v->nb[0]) % v->nb[1]);
            const int cz = (int)(b / ((long long)v->nb[0] * v->nb[1]));
            bool skip = true;
            for (int e = 0; e < 8; ++e) {
                const int x = cx + (e & 1), y = cy + ((e >> 1) & 1), z = cz + ((e >> 2) & 1);
                if (x < v->nb[0] && y < v->nb[1] && z < v->nb[2])
                    skip &= (v->h_flag[((long long)z * v->nb[1] + y) * v->nb[0] + x] & kFlagNoNeg) != 0;
            }
            v->h_flag[cflag_offset(nb) + b] = skip ? kCellSkip : 0;
            if (!skip) ++sup[((size_t)(cz / kSuper) * v->nsb[1] + cy / kSuper) * v->nsb[0] + cx / kSuper];
        }
        // neighbour counts of the super-brick words (see kSupCount)
        std::vector<unsigned> word(sup);
        for (int sz = 0; sz < v->nsb[2]; ++sz)
            for (int sy = 0; sy < v->nsb[1]; ++sy)
                for (int sx = 0; sx < v->nsb[0]; ++sx) {
                    if (!sup[((size_t)sz * v->nsb[1] + sy) * v->nsb[0] + sx]) continue;
                    for (int z = std::max(0, sz - kSupReach); z <= std::min(v->nsb[2] - 1, sz + kSupReach); ++z)
                        for (int y = std::max(0, sy - kSupReach); y <= std::min(v->nsb[1] - 1, sy + kSupReach); ++y)
                            for (int x = std::max(0, sx - kSupReach); x <= std::min(v->nsb[0] - 1, sx + kSupReach);
                                 ++x) {
                                const int d = std::max(std::abs(x - sx), std::max(std::abs(y - sy), std::abs(z - sz)));
                                word[((size_t)z * v->nsb[1] + y) * v->nsb[0] + x] +=
                                    (d <= 1 ? kSupNear1 : 0u) + kSupNear2;
                            }
                }
        std::memcpy(v->h_flag + super_offset(nb), word.data(), sizeof(unsigned) * word.size());
    }
    return MV_OK;
}

mv_status mv_read_brick_flags(mv_ctx *c, int32_t id, uint8_t *host_flags, uint64_t cap)
{
    if (!c || !host_flags) return fail(c, MV_ERR_ARG, "null argument");
    Volume *v;
    mv_status st = find_volume(c, id, &v);
    if (st) return st;
    if (cap < (uint64_t)v->nbricks) return fail(c, MV_ERR_ARG, "flag buffer too small");
    cudaSetDevice(c->device);
    st = wait_all(c);
    if (st) return st;
    if (v->ready_pending) MV_CUDA(c, cudaEventSynchronize(v->ready));
    if (v->resident)
        MV_CUDA(c, cudaMemcpy(host_flags, v->d_flag, (size_t)v->nbricks, cudaMemcpyDeviceToHost));
    else
        std::memcpy(host_flags, v->h_flag, (size_t)v->nbricks);
    return MV_OK;
}

mv_status mv_get_stats(mv_ctx *c, mv_stats *out, int32_t reset)
{
    if (!c || !out) return fail(c, MV_ERR_ARG, "null argument");
    cudaSetDevice(c->device);
    mv_status st = wait_all(c);
    if (st) return st;
    Stats h;
    MV_CUDA(c, cudaMemcpy(&h, c->d_stats, sizeof(Stats), cudaMemcpyDeviceToHost));
    out->swept = h.swept;
    out->updated = h.updated;
    out->band = h.band;
    out->bricks = h.bricks;
    out->rays = h.rays;
    out->ray_samples = h.ray_samples;
    out->ray_skips = h.ray_skips;
    out->ray_hits = h.ray_hits;
    out->stream_up = h.stream_up;
    out->stream_down = h.stream_down;
    if (reset) MV_CUDA(c, cudaMemset(c->d_stats, 0, sizeof(Stats)));
    return MV_OK;
}

mv_status mv_set_timing(mv_ctx *c, int32_t enable)
{
    if (!c) return MV_ERR_ARG;
    c->timing = enable != 0;
    return MV_OK;
}

mv_status mv_get_timings(mv_ctx *c, mv_timings *out, int32_t reset)
{
    if (!c || !out) return fail(c, MV_ERR_ARG, "null argument");
    cudaSetDevice(c->device);
    mv_status st = wait_all(c);
    if (st) return st;
    st = collect_timings(c);
    if (st) return st;
    for (int k = 0; k < MV_KERNEL_KINDS; ++k) {
        out->launches[k] = c->launches[k];
        out->ms[k] = c->ms[k];
        out->timed[k] = c->timed[k];
    }
    if (reset) {
        std::fill(c->launches, c->launches + MV_KERNEL_KINDS, 0);
        std::fill(c->ms, c->ms + MV_KERNEL_KINDS, 0.0);
        std::fill(c->timed, c->timed + MV_KERNEL_KINDS, 0);
    }
    return MV_OK;
}

mv_status mv_synchronize(mv_ctx *c)
{
    if (!c) return MV_ERR_ARG;
    cudaSetDevice(c->device);
    return wait_all(c);
}

}  // extern "C"
