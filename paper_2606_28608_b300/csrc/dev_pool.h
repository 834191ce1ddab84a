// dev_pool.h -- device buffers handed from one set-up of a plan to the next.
//
// pdmk_set_sources replaces every per-set-up array of a plan.  Instead of freeing the old
// arrays and allocating the new ones (each cudaFree synchronises the device, and the plan's
// arrays run to tens of GB), the old ones become spares: a request takes the smallest spare
// of at least its size and at most 5/4 of it plus 1 MiB, else it allocates.  Spares that no
// request took are freed when the set-up ends (trim), and all spares are freed before a
// failed allocation is retried, so a larger problem is never refused for want of memory that
// spares hold.  Buffers come back uninitialised, as from cudaMalloc.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <utility>
#include <vector>

namespace pdmk {

struct DevicePool {
    std::vector<std::pair<void*, size_t>> spare;  // (buffer, bytes)

    // a buffer of at least bytes, or nullptr (the CUDA error is cleared)
    void* get(size_t bytes) {
        if (bytes == 0) bytes = 1;
        size_t best = spare.size();
        for (size_t i = 0; i < spare.size(); ++i) {
            const size_t b = spare[i].second;
            if (b >= bytes && b <= bytes + bytes / 4 + (size_t(1) << 20) &&
                (best == spare.size() || b < spare[best].second))
                best = i;
        }
        if (best < spare.size()) {
            void* p = spare[best].first;
            spare.erase(spare.begin() + static_cast<std::ptrdiff_t>(best));
            return p;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) == cudaSuccess) return p;
        cudaGetLastError();
        trim();
        if (cudaMalloc(&p, bytes) == cudaSuccess) return p;
        cudaGetLastError();
        return nullptr;
    }
    void put(void* p, size_t bytes) {
        if (p) spare.push_back({p, bytes});
    }
    void trim() {
        for (auto& s : spare) cudaFree(s.first);
        spare.clear();
    }
};

}  // namespace pdmk
