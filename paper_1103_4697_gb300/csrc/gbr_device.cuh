// Device helpers shared by the kernel files of libgbres (internal).
#pragma once
#include <math.h>

#include <map>
#include <mutex>
#include <tuple>

#include "gbr_internal.h"

namespace gbr {

// i = w^(2^(kRootLog - 2)), a square root of -1 mod p, in Montgomery form: the
// entry T2[e / 128] of the root tables for e = 2^(kRootLog - 2) (T1[0] = R).
static_assert((kRootOrder / 4) % 128 == 0, "i must be an entry of the second root table");
__device__ __forceinline__ uint32_t iota_mont(const ResLaunch &L, int pidx) {
    return L.roots[(int64_t)pidx * kRootTabWords + 128 + (kRootOrder / 4) / 128];
}

// Point x_j of a quartic set in Montgomery form (index layout of quad_h).
__device__ __forceinline__ uint32_t quad_point_mont(int j, uint32_t iota_m, const ModP &M) {
    if (j == 0) return 0u;
    const int a = (j - 1) / 4 + 1, k = (j - 1) & 3;
    uint32_t x = mp_to((uint32_t)a, M);
    if (k & 1) x = mp_mul(x, iota_m, M);
    return (k & 2) ? mp_neg(x, M.p) : x;
}

// Entry j of the contraction operand of group `mode` (n points) from one pair's
// values v (Montgomery form, below p): GEMM_PLAIN v_j; GEMM_EVEN v(0) (j = 0) or
// v(j) + v(-j); GEMM_ODD v(j+1) - v(-(j+1)); GEMM_Q0 v(0) (j = 0) or
// sum_k v(i^k j); GEMM_Q0 + t (t = 1, 2, 3) sum_k i^(-k t) v(i^k (j+1)).  In two
// steps, so that a pipelined caller can keep the loads in flight: operand_loads
// fetches the (up to four) values, a quartic quadruple as one 16-byte load (v is
// 16-byte aligned for quartic pairs; the point 0 sits at 4 h = 4 (n - 1) for
// GEMM_Q0), operand_combine forms the entry (below p, in the values' form; iota is i
// in Montgomery form, read by the quartic modes only).
__device__ __forceinline__ void operand_loads(const uint32_t *v, int mode, int j, int n, uint32_t (&x)[4]) {
    x[1] = x[2] = x[3] = 0u;
    if (mode == GEMM_PLAIN) {
        x[0] = v[j];
    } else if (mode == GEMM_EVEN) {
        x[0] = v[j == 0 ? 0 : 2 * j - 1];
        if (j) x[1] = v[2 * j];
    } else if (mode == GEMM_ODD) {
        x[0] = v[2 * j + 1];
        x[1] = v[2 * j + 2];
    } else if (mode == GEMM_Q0 && j == 0) {
        x[0] = v[4 * (n - 1)];
    } else {
        const uint4 q = *reinterpret_cast<const uint4 *>(v + 4 * (mode == GEMM_Q0 ? j - 1 : j));
        x[0] = q.x;
        x[1] = q.y;
        x[2] = q.z;
        x[3] = q.w;
    }
}

__device__ __forceinline__ uint32_t operand_combine(const uint32_t (&x)[4], int mode, uint32_t iota, const ModP &M) {
    if (mode == GEMM_PLAIN) return x[0];
    if (mode == GEMM_EVEN) return mp_add(x[0], x[1], M.p);
    if (mode == GEMM_ODD) return mp_sub(x[0], x[1], M.p);
    const int t = mode - GEMM_Q0;
    if (t == 0) return mp_add(mp_add(x[0], x[2], M.p), mp_add(x[1], x[3], M.p), M.p);
    if (t == 2) return mp_sub(mp_add(x[0], x[2], M.p), mp_add(x[1], x[3], M.p), M.p);
    const uint32_t d = mp_sub(x[0], x[2], M.p), e = mp_mul(mp_sub(x[1], x[3], M.p), iota, M);
    return t == 1 ? mp_sub(d, e, M.p) : mp_add(d, e, M.p);
}

__device__ __forceinline__ uint32_t contraction_operand(const uint32_t *v, int mode, int j, int n, uint32_t iota,
                                                        const ModP &M) {
    uint32_t x[4];
    operand_loads(v, mode, j, n, x);
    return operand_combine(x, mode, iota, M);
}

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
