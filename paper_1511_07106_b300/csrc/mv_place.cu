// mv_place.cu -- dynamic volume placement (Sec. Dynamic Mapping for SLAM;
// Sec. Insertion and Removal).
//
// Every frame the ray endpoints of the valid depth pixels are binned into a
// lattice of cells, one cell per possible volume origin h_t = k (d_v - 2);
// the count c(l) per cell drives which volumes are resident.  The binning is
// one kernel over the pixels (FP64 endpoint, warp-aggregated inserts into an
// open-addressing table) and one compaction kernel; the policy itself is a
// few dozen cells on the host and acts through the public C API (add, swap
// out, swap in).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "mvtsdf.h"

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr long long kCellRange = 1ll << 20;  // |cell coordinate| < 2^20 (21-bit fields)

struct Pose16 {
    double m[16];
};

__device__ __forceinline__ unsigned long long pack_cell(long long x, long long y, long long z)
{
    return (unsigned long long)(x + kCellRange) | ((unsigned long long)(y + kCellRange) << 21) |
           ((unsigned long long)(z + kCellRange) << 42);
}

__device__ __forceinline__ unsigned hash_key(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return (unsigned)k;
}

// One thread per pixel.  The endpoint is evaluated in FP64 with explicitly
// rounded operations (no contraction), in a fixed order:
//   xn = (x - cx) / fx, yn = (y - cy) / fy, p = (D xn, D yn, D),
//   e_a = ((R_a0 p_0 + R_a1 p_1) + R_a2 p_2) + t_a, l_a = floor(e_a / cell_m).
// Lanes of a warp with the same cell insert once, with their number.
__global__ void __launch_bounds__(256) endpoint_hist_kernel(const float *__restrict__ depth, int W, int H,
                                                            double fx, double fy, double cx, double cy,
                                                            Pose16 T, double cell_m, float z_min, float z_max,
                                                            unsigned long long *__restrict__ keys,
                                                            unsigned *__restrict__ counts, unsigned mask,
                                                            unsigned *__restrict__ flags)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = kEmpty;
    if (p < (long long)W * H) {
        const float Df = __ldg(depth + p);
        if (Df > 0.f && Df >= z_min && Df <= z_max) {
            const int x = (int)(p % W), y = (int)(p / W);
            const double D = (double)Df;
            const double xn = __ddiv_rn(__dsub_rn((double)x, cx), fx);
            const double yn = __ddiv_rn(__dsub_rn((double)y, cy), fy);
            const double pc0 = __dmul_rn(D, xn), pc1 = __dmul_rn(D, yn), pc2 = D;
            long long c[3];
            bool ok = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double e = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(T.m[4 * a], pc0), __dmul_rn(T.m[4 * a + 1], pc1)),
                                                     __dmul_rn(T.m[4 * a + 2], pc2)),
                                           T.m[4 * a + 3]);
                const double q = floor(__ddiv_rn(e, cell_m));
                ok &= q >= (double)-kCellRange && q < (double)kCellRange;
                c[a] = ok ? (long long)q : 0;
            }
            if (ok) key = pack_cell(c[0], c[1], c[2]);
            else atomicOr(flags, 1u);
        }
    }
    const unsigned same = __match_any_sync(0xffffffffu, key);
    if ((int)(threadIdx.x & 31) != __ffs(same) - 1 || key == kEmpty) return;
    unsigned h = hash_key(key) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(keys + h, kEmpty, key);
        if (prev == kEmpty || prev == key) {
            atomicAdd(counts + h, (unsigned)__popc(same));
            return;
        }
        h = (h + 1) & mask;
    }
    atomicOr(flags, 2u);  // table full
}

__global__ void __launch_bounds__(256) compact_hist_kernel(const unsigned long long *__restrict__ keys,
                                                           const unsigned *__restrict__ counts, unsigned n,
                                                           unsigned long long *__restrict__ out_keys,
                                                           unsigned *__restrict__ out_counts,
                                                           unsigned *__restrict__ n_out)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        if (k == kEmpty) continue;
        const unsigned j = atomicAdd(n_out, 1u);
        out_keys[j] = k;
        out_counts[j] = counts[i];
    }
}

using Cell = std::array<int, 3>;

// (z, y, x) order of cells
bool cell_less(const Cell &a, const Cell &b)
{
    if (a[2] != b[2]) return a[2] < b[2];
    if (a[1] != b[1]) return a[1] < b[1];
    return a[0] < b[0];
}

struct CellLess {
    bool operator()(const Cell &a, const Cell &b) const { return cell_less(a, b); }
};

}  // namespace

struct mv_placer {
    mv_ctx *ctx = nullptr;
    mv_placement_config cfg{};
    float z_min = 0.f, z_max = INFINITY;
    int device = 0;
    // device table (capacity a power of two >= 2 x pixels) and its compaction
    unsigned long long *d_keys = nullptr, *d_out_keys = nullptr;
    unsigned *d_counts = nullptr, *d_out_counts = nullptr, *d_meta = nullptr;  // meta: n_out, flags
    unsigned cap = 0;
    // placed volumes by cell, resident or swapped out
    std::map<Cell, int, CellLess> id_of;
    std::string err;
};

namespace {

mv_status pfail(mv_placer *p, mv_status st, const std::string &msg)
{
    if (p) p->err = msg;
    return st;
}

mv_status pcuda(mv_placer *p, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return MV_OK;
    cudaGetLastError();
    return pfail(p, e == cudaErrorMemoryAllocation ? MV_ERR_OOM : MV_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define PL_CUDA(p, call)                                           \
    do {                                                           \
        const mv_status st_ = pcuda((p), (call), #call);           \
        if (st_ != MV_OK) return st_;                              \
    } while (0)

bool valid_view(const mv_intrinsics *K, const double *T)
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

// c(l) of one frame, sorted by cell (z, y, x).
mv_status histogram(mv_placer *p, const float *depth, const mv_intrinsics *K, const double T[16],
                    std::vector<Cell> &cells, std::vector<unsigned> &counts, cudaStream_t s)
{
    if (!depth || !valid_view(K, T)) return pfail(p, MV_ERR_ARG, "bad frame arguments");
    if (reinterpret_cast<uintptr_t>(depth) & 3u) return pfail(p, MV_ERR_ARG, "depth must be 4-byte aligned");
    cudaSetDevice(p->device);
    const long long npx = (long long)K->width * K->height;
    unsigned need = 1024;
    while ((long long)need < 2 * npx) need <<= 1;
    if (need > p->cap) {
        cudaFree(p->d_keys);
        cudaFree(p->d_counts);
        cudaFree(p->d_out_keys);
        cudaFree(p->d_out_counts);
        p->d_keys = p->d_out_keys = nullptr;
        p->d_counts = p->d_out_counts = nullptr;
        p->cap = 0;
        PL_CUDA(p, cudaMalloc((void **)&p->d_keys, sizeof(unsigned long long) * need));
        PL_CUDA(p, cudaMalloc((void **)&p->d_counts, sizeof(unsigned) * need));
        PL_CUDA(p, cudaMalloc((void **)&p->d_out_keys, sizeof(unsigned long long) * need));
        PL_CUDA(p, cudaMalloc((void **)&p->d_out_counts, sizeof(unsigned) * need));
        p->cap = need;
    }
    if (!p->d_meta) PL_CUDA(p, cudaMalloc((void **)&p->d_meta, sizeof(unsigned) * 2));
    PL_CUDA(p, cudaMemsetAsync(p->d_keys, 0xFF, sizeof(unsigned long long) * p->cap, s));
    PL_CUDA(p, cudaMemsetAsync(p->d_counts, 0, sizeof(unsigned) * p->cap, s));
    PL_CUDA(p, cudaMemsetAsync(p->d_meta, 0, sizeof(unsigned) * 2, s));
    Pose16 Tm;
    for (int i = 0; i < 16; ++i) Tm.m[i] = T[i];
    const double cell_m = (double)p->cfg.cell_voxels * (double)p->cfg.voxel_size;
    const unsigned blocks = (unsigned)((npx + 255) / 256);
    endpoint_hist_kernel<<<blocks, 256, 0, s>>>(depth, K->width, K->height, (double)K->fx, (double)K->fy,
                                                (double)K->cx, (double)K->cy, Tm, cell_m, p->z_min, p->z_max,
                                                p->d_keys, p->d_counts, p->cap - 1, p->d_meta + 1);
    PL_CUDA(p, cudaGetLastError());
    compact_hist_kernel<<<256, 256, 0, s>>>(p->d_keys, p->d_counts, p->cap, p->d_out_keys, p->d_out_counts,
                                            p->d_meta);
    PL_CUDA(p, cudaGetLastError());
    unsigned meta[2] = {0u, 0u};
    PL_CUDA(p, cudaMemcpyAsync(meta, p->d_meta, sizeof(meta), cudaMemcpyDeviceToHost, s));
    PL_CUDA(p, cudaStreamSynchronize(s));
    if (meta[1] & 1u) return pfail(p, MV_ERR_CAPACITY, "an endpoint cell coordinate is beyond +-2^20");
    if (meta[1] & 2u) return pfail(p, MV_ERR_CAPACITY, "endpoint table full");
    std::vector<unsigned long long> k(meta[0]);
    std::vector<unsigned> c(meta[0]);
    if (meta[0]) {
        PL_CUDA(p, cudaMemcpyAsync(k.data(), p->d_out_keys, sizeof(unsigned long long) * meta[0],
                                   cudaMemcpyDeviceToHost, s));
        PL_CUDA(p, cudaMemcpyAsync(c.data(), p->d_out_counts, sizeof(unsigned) * meta[0], cudaMemcpyDeviceToHost,
                                   s));
        PL_CUDA(p, cudaStreamSynchronize(s));
    }
    std::vector<std::pair<Cell, unsigned>> all(meta[0]);
    const unsigned long long m21 = (1ull << 21) - 1;
    for (unsigned i = 0; i < meta[0]; ++i) {
        const Cell cl = {(int)((long long)(k[i] & m21) - kCellRange), (int)((long long)((k[i] >> 21) & m21) - kCellRange),
                         (int)((long long)((k[i] >> 42) & m21) - kCellRange)};
        all[i] = {cl, c[i]};
    }
    std::sort(all.begin(), all.end(), [](const auto &a, const auto &b) { return cell_less(a.first, b.first); });
    cells.resize(all.size());
    counts.resize(all.size());
    for (size_t i = 0; i < all.size(); ++i) {
        cells[i] = all[i].first;
        counts[i] = all[i].second;
    }
    return MV_OK;
}

}  // namespace

extern "C" {

mv_status mv_placer_create(mv_ctx *ctx, const mv_placement_config *cfg, mv_placer **out)
{
    if (!out) return MV_ERR_ARG;
    *out = nullptr;
    if (!ctx || !cfg) return MV_ERR_ARG;
    if (cfg->cell_voxels < 1 || cfg->volume_voxels < 2 || cfg->volume_voxels < cfg->cell_voxels ||
        cfg->volume_voxels > 8192 || !(cfg->voxel_size > 0.f) || !std::isfinite(cfg->voxel_size) ||
        cfg->max_volumes < 1 || !(cfg->hysteresis >= 1.f) || !std::isfinite(cfg->hysteresis) ||
        cfg->min_count < 1 || cfg->fmt < MV_TSDF_F32 || cfg->fmt > MV_TSDF_I16)
        return MV_ERR_ARG;
    mv_config mc;
    if (mv_get_config(ctx, &mc) != MV_OK) return MV_ERR_ARG;
    mv_placer *p = new mv_placer();
    p->ctx = ctx;
    p->cfg = *cfg;
    p->z_min = mc.z_min;
    p->z_max = mc.z_max;
    p->device = mv_get_device(ctx);
    *out = p;
    return MV_OK;
}

mv_status mv_placer_destroy(mv_placer *p)
{
    if (!p) return MV_OK;
    cudaSetDevice(p->device);
    cudaFree(p->d_keys);
    cudaFree(p->d_counts);
    cudaFree(p->d_out_keys);
    cudaFree(p->d_out_counts);
    cudaFree(p->d_meta);
    delete p;
    return MV_OK;
}

const char *mv_placer_last_error(const mv_placer *p)
{
    return p ? p->err.c_str() : "null placer";
}

mv_status mv_placer_histogram(mv_placer *p, const float *depth, const mv_intrinsics *K, const double T[16],
                              int32_t *cells, uint32_t *counts, int32_t cap, int32_t *n, void *stream)
{
    if (!p) return MV_ERR_ARG;
    if (!n || cap < 0 || (cap > 0 && (!cells || !counts))) return pfail(p, MV_ERR_ARG, "bad output arguments");
    std::vector<Cell> cl;
    std::vector<unsigned> cn;
    const mv_status st = histogram(p, depth, K, T, cl, cn, (cudaStream_t)stream);
    if (st) return st;
    *n = (int32_t)cl.size();
    const size_t m = std::min(cl.size(), (size_t)cap);
    for (size_t i = 0; i < m; ++i) {
        cells[3 * i] = cl[i][0];
        cells[3 * i + 1] = cl[i][1];
        cells[3 * i + 2] = cl[i][2];
        counts[i] = cn[i];
    }
    return cl.size() > (size_t)cap ? pfail(p, MV_ERR_CAPACITY, "more cells than cap") : MV_OK;
}

mv_status mv_placer_update(mv_placer *p, const float *depth, const mv_intrinsics *K, const double T[16],
                           mv_placement_result *out, void *stream)
{
    if (!p) return MV_ERR_ARG;
    std::vector<Cell> cl;
    std::vector<unsigned> cn;
    mv_status st = histogram(p, depth, K, T, cl, cn, (cudaStream_t)stream);
    if (st) return st;
    std::map<Cell, unsigned, CellLess> hist;
    for (size_t i = 0; i < cl.size(); ++i) hist[cl[i]] = cn[i];
    auto count = [&](const Cell &c) -> unsigned {
        auto it = hist.find(c);
        return it == hist.end() ? 0u : it->second;
    };
    // the registry as the context sees it now (volumes removed by the caller are forgotten)
    std::vector<Cell> resident;
    for (auto it = p->id_of.begin(); it != p->id_of.end();) {
        mv_volume_info q;
        if (mv_query(p->ctx, it->second, &q) != MV_OK) {
            it = p->id_of.erase(it);
            continue;
        }
        if (q.resident) resident.push_back(it->first);
        ++it;
    }
    // candidates: non-resident cells with enough endpoints, by decreasing
    // count, ties by increasing (z, y, x)
    std::vector<Cell> cand;
    for (size_t i = 0; i < cl.size(); ++i) {
        if (cn[i] < (unsigned)p->cfg.min_count) continue;
        if (std::find(resident.begin(), resident.end(), cl[i]) != resident.end()) continue;
        cand.push_back(cl[i]);
    }
    std::stable_sort(cand.begin(), cand.end(), [&](const Cell &a, const Cell &b) { return count(a) > count(b); });
    std::vector<Cell> enter, leave;
    size_t i = 0;
    while (i < cand.size() && (int)resident.size() < p->cfg.max_volumes) {
        resident.push_back(cand[i]);
        enter.push_back(cand[i]);
        ++i;
    }
    for (; i < cand.size() && !resident.empty(); ++i) {
        // the resident cell with the lowest count, ties by increasing (z, y, x)
        size_t lo = 0;
        for (size_t r = 1; r < resident.size(); ++r) {
            const unsigned a = count(resident[r]), b = count(resident[lo]);
            if (a < b || (a == b && cell_less(resident[r], resident[lo]))) lo = r;
        }
        if (!((double)count(cand[i]) > (double)p->cfg.hysteresis * (double)count(resident[lo]))) break;
        const Cell gone = resident[lo];
        resident.erase(resident.begin() + (long)lo);
        // a cell that entered in this step and leaves again is simply not added
        auto e = std::find(enter.begin(), enter.end(), gone);
        if (e != enter.end()) enter.erase(e); else leave.push_back(gone);
        resident.push_back(cand[i]);
        enter.push_back(cand[i]);
    }
    mv_placement_result r{(int32_t)cl.size(), 0, 0, 0, 0};
    for (const Cell &c : leave) {
        st = mv_swap_out(p->ctx, p->id_of.at(c), stream);
        if (st) return pfail(p, st, std::string("swap out: ") + mv_last_error(p->ctx));
        ++r.evicted;
    }
    for (const Cell &c : enter) {
        auto it = p->id_of.find(c);
        if (it != p->id_of.end()) {
            st = mv_swap_in(p->ctx, it->second, stream);
            if (st) return pfail(p, st, std::string("swap in: ") + mv_last_error(p->ctx));
            ++r.restored;
        } else {
            mv_volume_desc d{};
            for (int a = 0; a < 3; ++a) {
                d.h_t[a] = c[a] * p->cfg.cell_voxels;
                d.h_r[a] = p->cfg.volume_voxels;
            }
            d.voxel_size = p->cfg.voxel_size;
            d.fmt = (mv_tsdf_fmt)p->cfg.fmt;
            int32_t id = -1;
            st = mv_add_volume(p->ctx, &d, &id);
            if (st) return pfail(p, st, std::string("add volume: ") + mv_last_error(p->ctx));
            p->id_of[c] = id;
            ++r.added;
        }
    }
    r.resident = (int32_t)resident.size();
    if (out) *out = r;
    return MV_OK;
}

mv_status mv_placer_list(mv_placer *p, int32_t *ids, int32_t *cells, int32_t *resident, int32_t cap, int32_t *n)
{
    if (!p) return MV_ERR_ARG;
    if (!n || cap < 0 || (cap > 0 && (!ids || !cells || !resident)))
        return pfail(p, MV_ERR_ARG, "bad output arguments");
    std::vector<std::pair<int, Cell>> v;
    for (auto &kv : p->id_of) v.push_back({kv.second, kv.first});
    std::sort(v.begin(), v.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    int32_t k = 0;
    for (auto &e : v) {
        mv_volume_info q;
        if (mv_query(p->ctx, e.first, &q) != MV_OK) continue;
        if (k < cap) {
            ids[k] = e.first;
            cells[3 * k] = e.second[0];
            cells[3 * k + 1] = e.second[1];
            cells[3 * k + 2] = e.second[2];
            resident[k] = q.resident;
        }
        ++k;
    }
    *n = k;
    return MV_OK;
}

}  // extern "C"
