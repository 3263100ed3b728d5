// Chinese remaindering that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need a result:
// a host that budgets every byte of GPU memory up front and forbids later
// allocations, code running inside another framework's memory pool or
// allocator callback, or a latency-critical loop where cudaMalloc/cudaFree
// would stall on an implicit device synchronisation.  For them
// gbr_crt_noalloc runs the same Garner reconstruction as the library's own CRT
// stage, but keeps its working digits in the fixed array below instead of in
// memory the library allocates.  The caller supplies the residues and the
// output buffers; nothing else is allocated by this file, ever.
#include <algorithm>
#include <mutex>

#include "gbr_core.h"

namespace gbr {

// Fixed working storage for the Garner digits of every call: one word per
// (coefficient, prime).  Loaded with the library and held on every GPU that
// loads it until the process exits.  Calls share it, so two calls whose
// kernels overlap on the GPU (different streams, or different host threads)
// overwrite each other's digits: serialise them.  Nothing in it has to start
// at zero (each digit is written before it is read).
constexpr int64_t kNoallocScratchWords = int64_t(1) << 20;   // 4 MiB
static __device__ __align__(256) uint32_t g_crt_scratch[kNoallocScratchWords];

struct NoallocPrimes {
    ModP m[GBR_NOALLOC_MAX_PRIMES];
};

// Same reconstruction as k_crt: Garner digits v_i (kept in `digits`, not in the
// residue input), symmetric lift by comparing the digits with (p_i - 1)/2 from
// the top, and Horner evaluation of the magnitude into 32-bit limbs written
// straight into the caller's output.  The Garner constants for the prefix prime
// list are rebuilt by each block in shared memory.
__global__ void k_crt_noalloc(const uint32_t *res, int k, int ncoef, int64_t stride, uint32_t *mag, int limbs,
                              int8_t *sign, uint32_t *digits, NoallocPrimes P) {
    __shared__ uint32_t cinv[GBR_NOALLOC_MAX_PRIMES];
    __shared__ uint32_t pm[GBR_NOALLOC_MAX_PRIMES * (GBR_NOALLOC_MAX_PRIMES - 1) / 2];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const ModP M = P.m[i];
        uint32_t prod = M.r1;
        for (int j = 0; j < i; ++j) {
            uint32_t pj = P.m[j].p;
            pj = min(pj, pj - M.p);
            uint32_t pjm = mp_to(pj, M);
            pm[i * (i - 1) / 2 + j] = pjm;
            prod = mp_mul(prod, pjm, M);
        }
        cinv[i] = mp_inv(prod, M);
    }
    __syncthreads();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncoef; c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t *v = digits + c * k;
        v[0] = res[c];
        for (int i = 1; i < k; ++i) {
            const ModP M = P.m[i];
            const uint32_t *pmi = pm + i * (i - 1) / 2;
            uint32_t t = v[i - 1];
            t = min(t, t - M.p);
            for (int j = i - 2; j >= 0; --j) {
                uint32_t vj = v[j];
                vj = min(vj, vj - M.p);
                t = mp_add(mp_mul(t, pmi[j], M), vj, M.p);
            }
            v[i] = mp_mul(mp_sub(res[(int64_t)i * stride + c], t, M.p), cinv[i], M);
        }
        int cmp = 0;
        for (int i = k - 1; i >= 0 && cmp == 0; --i) {
            uint32_t h = (P.m[i].p - 1u) >> 1;
            cmp = (v[i] > h) - (v[i] < h);
        }
        const bool neg = cmp > 0;
        uint32_t *o = mag + c * limbs;
        int nl = 0;
        for (int i = k - 1; i >= 0; --i) {
            const uint32_t p = P.m[i].p;
            uint32_t d = neg ? p - 1u - v[i] : v[i];
            uint32_t carry = d;
            for (int l = 0; l < nl; ++l) {
                uint64_t t = (uint64_t)o[l] * p + carry;
                o[l] = (uint32_t)t;
                carry = (uint32_t)(t >> 32);
            }
            if (carry) o[nl++] = carry;
        }
        if (neg) {
            int l = 0;
            for (; l < nl; ++l)
                if (++o[l] != 0u) break;
            if (l == nl) o[nl++] = 1u;
        }
        for (int l = nl; l < limbs; ++l) o[l] = 0u;
        sign[c] = nl == 0 ? 0 : (neg ? -1 : 1);
    }
}

// Device address of g_crt_scratch, looked up once per device with that device
// current (the host-side name of a __device__ array is only a stand-in).
static std::mutex g_scratch_mu;
static uint32_t *g_scratch_ptr[64];
static bool g_scratch_ready[64];

static cudaError_t scratch_for_current_device(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_ready[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_crt_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (uint32_t *)p;
        g_scratch_ready[dev] = true;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace gbr

using namespace gbr;

extern "C" int gbr_crt_noalloc(const uint32_t *residues, int k, int ncoef, int64_t stride, uint32_t *mag, int limbs,
                               int8_t *sign, void *stream) {
    if (!residues || !mag || !sign || k < 1 || ncoef < 0 || stride < ncoef) return GBR_EINVAL;
    if (k > GBR_NOALLOC_MAX_PRIMES) return GBR_ELIMIT;
    if ((int64_t)ncoef * k > kNoallocScratchWords) return GBR_ELIMIT;
    if (limbs < (31 * k + 31) / 32) return GBR_EINVAL;
    if (ncoef == 0) return GBR_OK;
    uint32_t *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return GBR_EDEVICE;
    NoallocPrimes P;
    const ModP *hm = host_mods();
    for (int i = 0; i < k; ++i) P.m[i] = hm[i];
    const int block = 128;
    int grid = (int)std::min<int64_t>((ncoef + block - 1) / block, 1184);
    k_crt_noalloc<<<grid, block, 0, (cudaStream_t)stream>>>(residues, k, ncoef, stride, mag, limbs, sign, scratch, P);
    return cudaGetLastError() == cudaSuccess ? GBR_OK : GBR_EDEVICE;
}
