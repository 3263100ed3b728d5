// Interpolation at roots of unity (step A4, NTT form).
//
// Every table prime is 1 mod 2^kRootLog, so it has a root of unity w of order
// 2^kRootLog.  A pair planned with root points (PairPlan::sym == PTS_ROOTS) is
// evaluated at x_j = u^j, j = 0..N-1, with N = Pe a power of two at least the
// number of coefficients P and u = w^(2^kRootLog / N) a primitive N-th root of
// unity.  The coefficients of R mod p are then the inverse discrete Fourier
// transform of the values:
//     c_k = N^-1 sum_j R(u^j) u^(-j k),   k = 0..N-1,
// and c_k = 0 for k >= P (the degree bound), which the kernel checks.  The
// transform is the radix-2 decimation-in-frequency butterfly network
// (Gentleman-Sande) on the values in natural order, which leaves N c_k at the
// bit-reversed position of k; O(N log N) Montgomery products per (pair, prime)
// instead of the O(N^2) of an inverse-Vandermonde contraction or of Newton.
//
// One CTA per (pair, prime) item of the work list: the values and the N/2
// twiddles u^(-t) (built from the prime's root table) in shared memory, one
// barrier per stage.
#include "gbr_device.cuh"

namespace gbr {

__global__ void __launch_bounds__(256) k_interp_ntt(ResLaunch L, WorkList w) {
    if (stage_skipped(L)) return;
    extern __shared__ uint32_t ns[];
    for (int64_t item = blockIdx.x; item < w.total; item += gridDim.x) {
        const int bi = wl_find(w.start, w.n, item);
        const PairPlan &P = L.plan[w.pairs[bi]];
        const int i = (int)(item - w.start[bi]);
        const int pidx = prime_of(P, L.pmap, i);
        const ModP M = L.mods[pidx];
        const uint32_t *rt = L.roots + (int64_t)pidx * kRootTabWords;
        const int N = P.Pe;
        const int lg = 31 - __clz(N);
        const int s = kRootOrder >> lg;          // u = w^s
        uint32_t *a = ns;                        // N values
        uint32_t *tw = ns + N;                   // tw[t] = u^(-t) R mod p, t < N/2
        const uint32_t *v = L.val + P.val_off + (int64_t)i * N;
        for (int t = threadIdx.x; t < N; t += blockDim.x) a[t] = v[t];
        for (int t = threadIdx.x; t < N / 2; t += blockDim.x)
            tw[t] = root_pow(rt, (kRootOrder - s * t) & (kRootOrder - 1), M);
        __syncthreads();
        // stage with half-length h: blocks of 2h, butterfly t of a block uses u^(-t N / (2h))
        for (int h = N >> 1, st = 1; h >= 1; h >>= 1, st <<= 1) {
            for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
                const int t = b & (h - 1);
                const int x = ((b - t) << 1) + t;
                const uint32_t u0 = a[x], u1 = a[x + h];
                a[x] = mp_add(u0, u1, M.p);
                a[x + h] = mp_mul(mp_sub(u0, u1, M.p), tw[t * st], M);
            }
            __syncthreads();
        }
        // c_k = a[rev(k)] / N in normal form: a is Montgomery, N^-1 = p - (p - 1) / N plain
        const uint32_t ninv = M.p - (M.p - 1u) / (uint32_t)N;
        uint32_t *cf = L.cf + P.cf_off + (int64_t)i * P.P;
        bool high = false;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            const uint32_t c = mp_mul(a[__brev((unsigned)k) >> (32 - lg)], ninv, M);
            if (k < P.P) cf[k] = c;
            else high = high || c != 0u;
        }
        if (__syncthreads_or(high) && threadIdx.x == 0) atomicExch(L.err, kErrNttDegree);
    }
}

cudaError_t launch_interp_ntt(const ResLaunch &L, const WorkList &w, int maxN, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    const size_t smem = (size_t)(maxN + maxN / 2) * sizeof(uint32_t);
    if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
    const int block = maxN >= 512 ? 256 : std::max(32, maxN / 2);
    const int grid = persistent_grid(k_interp_ntt, block, smem, w.total);
    k_interp_ntt<<<grid, block, smem, s>>>(L, w);
    return cudaGetLastError();
}

cudaError_t configure_interp_ntt_kernel() {
    return cudaFuncSetAttribute(k_interp_ntt, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

}  // namespace gbr
