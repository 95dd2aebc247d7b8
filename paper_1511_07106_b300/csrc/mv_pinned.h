// mv_pinned.h -- a pool of pinned (page-locked, device-mapped) host buffers.
//
// Moving a volume out of GPU memory needs pinned host buffers; pinning a
// gigabyte takes a large fraction of a second, so a volume evicted for the
// first time stalls its frame.  The pool holds spare buffers of given sizes,
// pinned ahead of time on request (mv_reserve_host), and takes back the
// buffers of removed volumes while it holds fewer spares than reserved.
#pragma once

#include <cstddef>
#include <map>
#include <vector>

namespace mv {

class PinnedPool {
public:
    PinnedPool() = default;
    ~PinnedPool();
    PinnedPool(const PinnedPool &) = delete;
    PinnedPool &operator=(const PinnedPool &) = delete;

    // A spare buffer of exactly `bytes`, else a new allocation (nullptr when
    // that fails).
    void *take(size_t bytes);
    // Back to the spares while fewer than reserved are held, else freed.
    void give(void *p, size_t bytes);
    // Hold at least `count` spares of `bytes`, pinning the missing ones now;
    // spares above `count` are freed.  False when pinning fails.
    bool reserve(size_t bytes, int count);

private:
    std::map<size_t, std::vector<void *>> spare_;
    std::map<size_t, int> target_;
};

}  // namespace mv
