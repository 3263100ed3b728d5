// Device helpers shared by the kernel files of libgbres (internal).
#pragma once
#include <math.h>

#include <map>
#include <mutex>
#include <tuple>

#include "gbr_internal.h"

namespace gbr {

__device__ __forceinline__ int wl_find(const int64_t *start, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}


// SM count of the current device (queried once).
inline int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Occupancy per (kernel, block size, shared memory), queried once: launches that
// are being captured into a CUDA graph then make no query.
inline std::mutex g_occ_mu;
inline std::map<std::tuple<const void *, int, size_t>, int> g_occ;

template <typename K>
inline int persistent_grid(K kernel, int block, size_t smem, int64_t items_in_blocks) {
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> g(g_occ_mu);
        auto key = std::make_tuple((const void *)kernel, block, smem);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) {
            per_sm = it->second;
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
            g_occ[key] = per_sm;
        }
    }
    if (per_sm < 1) per_sm = 1;
    int64_t cap = (int64_t)per_sm * sm_count();
    return (int)(items_in_blocks < cap ? (items_in_blocks < 1 ? 1 : items_in_blocks) : cap);
}


}  // namespace gbr
