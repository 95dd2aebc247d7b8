// mv_pinned.cu -- pinned host buffer pool (see mv_pinned.h).
#include <cuda_runtime.h>

#include "mv_pinned.h"

namespace mv {

namespace {
void *alloc_pinned(size_t bytes)
{
    void *p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
}  // namespace

PinnedPool::~PinnedPool()
{
    for (auto &kv : spare_)
        for (void *p : kv.second) cudaFreeHost(p);
}

void *PinnedPool::take(size_t bytes)
{
    auto it = spare_.find(bytes);
    if (it != spare_.end() && !it->second.empty()) {
        void *p = it->second.back();
        it->second.pop_back();
        return p;
    }
    return alloc_pinned(bytes);
}

void PinnedPool::give(void *p, size_t bytes)
{
    if (!p) return;
    auto t = target_.find(bytes);
    if (t != target_.end() && (int)spare_[bytes].size() < t->second) {
        spare_[bytes].push_back(p);
        return;
    }
    cudaFreeHost(p);
}

bool PinnedPool::reserve(size_t bytes, int count)
{
    target_[bytes] = count < 0 ? 0 : count;
    auto &v = spare_[bytes];
    while ((int)v.size() > target_[bytes]) {
        cudaFreeHost(v.back());
        v.pop_back();
    }
    while ((int)v.size() < target_[bytes]) {
        void *p = alloc_pinned(bytes);
        if (!p) return false;
        v.push_back(p);
    }
    return true;
}

}  // namespace mv
