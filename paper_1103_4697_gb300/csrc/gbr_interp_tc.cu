// Interpolation (step A4) as an exact contraction on the tensor cores (tcgen05,
// bf16 operands, fp32 accumulators in tensor memory).
//
// For one prime p, one group of pairs and one inverse-Vandermonde matrix V
// (n x n, normal form) the coefficients are C[q][r] = sum_j X[q][j] V[r][j] with
// X the Montgomery-form operand of pair q (values, or the sums / differences of
// the values at +-i), so C = R coef (mod p).  Both operands are below p < 2^31
// and are split into four balanced base-256 digits in [-128, 127]:
// x = sum_s x_s 256^s.  A bf16 holds such a digit exactly, the product of two
// digits is at most 2^14, and the diagonal sums
//   D_u = sum_{s+t=u} X_s V_t^T     (u = 0..6, at most four digit pairs)
// over n <= 256 terms stay below 2^24 in magnitude, so fp32 accumulation is
// exact.  C = sum_u 256^u D_u is then formed exactly in 64-bit integers and
// reduced: coef = C R^-1 mod p.
//
// Tile: 128 pairs (tensor-memory lanes) x 64 coefficients (columns); the seven
// diagonals take 7 x 64 of the 512 tensor-memory columns.  The K dimension runs
// in chunks of 32 through two shared-memory stages: the CTA's threads (four per
// pair) split the operands into digits while thread 0 issues the 32 MMAs
// (16 digit pairs x 2 k-steps of 16) of the previous stage; tcgen05.commit
// releases a stage when its MMAs have read it.  When the operand's whole K
// extent fits (at most kTcResidentChunks chunks) its digits stay in shared memory
// and one CTA computes every row tile of the matrix against them, streaming only
// the matrix tiles, so the operand is loaded and split once instead of once per
// row tile.  Operand tiles use the
// no-swizzle K-major layout: core matrices of 8 rows x 8 elements (128 bytes),
// consecutive along K (LBO = 128 B), row groups 512 B apart (SBO).  The matrix
// digits are prepared once per cached matrix (k_vinv_tc) in exactly that layout.
#include "gbr_device.cuh"

namespace gbr {

constexpr int TC_M = 128;            // pairs per tile
constexpr int TC_N = 64;             // coefficients per tile
constexpr int TC_KC = 32;            // K per stage
constexpr int TC_DIAG = 7;
constexpr uint32_t TC_LBO = 128, TC_SBO = 512;
constexpr int TC_XPLANE = TC_M * TC_KC * 2;        // bytes of one digit plane of the operand tile
constexpr int TC_VPLANE = TC_N * TC_KC * 2;        // bytes of one digit plane of the matrix tile
constexpr int TC_XSLOT = 4 * TC_XPLANE;                   // 32 KB: the four digit planes of one chunk
constexpr int TC_VSLOT = 4 * TC_VPLANE;                   // 16 KB
constexpr int TC_RAW = TC_M * 33 * 4;                     // raw operand rows of one chunk
static_assert(kTcResidentChunks * TC_KC == kTcResidentN, "resident operand size");
constexpr int TC_VTILE_WORDS = 4 * TC_VPLANE / 4;         // uint32 words of one prepared matrix tile
constexpr int TC_THREADS = 512;                           // 16 warps share the staging of each chunk
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_PER_ROW = TC_THREADS / TC_M;             // threads per operand row (tensor-memory lane)
constexpr int TC_KG = TC_KC / 8 / TC_PER_ROW;             // K groups of 8 each thread splits per chunk
constexpr int TC_CPT = TC_N / TC_PER_ROW;                 // epilogue columns per thread
static_assert(TC_KG >= 1 && TC_CPT % 4 == 0 && TC_M % TC_WARPS == 0, "staging split");

// element (r, k) of a rows x 32 digit plane, in bf16 units
__host__ __device__ inline int tc_elem(int r, int k) { return (r >> 3) * 256 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7); }

// balanced base-256 digits of x < 2^31 as bf16 bit patterns: y = x + 0x808080
// carries each of the lower three digits into [0, 255] + 128; a digit d in
// [0, 255] becomes the float 2^23 + d exactly (bit pattern 0x4B0000dd), from
// which 2^23 + 128 is subtracted exactly; the top digit (below 128) likewise
// with 2^23.  An exact small integer's bf16 is the float's upper half.
__device__ __forceinline__ void tc_digits(uint32_t x, uint32_t &d0, uint32_t &d1, uint32_t &d2, uint32_t &d3) {
    const uint32_t y = x + 0x808080u;
    const float f0 = __uint_as_float(__byte_perm(y, 0x4B000000u, 0x7650)) - 8388736.0f;
    const float f1 = __uint_as_float(__byte_perm(y, 0x4B000000u, 0x7651)) - 8388736.0f;
    const float f2 = __uint_as_float(__byte_perm(y, 0x4B000000u, 0x7652)) - 8388736.0f;
    const float f3 = __uint_as_float(__byte_perm(y, 0x4B000000u, 0x7653)) - 8388608.0f;
    d0 = __float_as_uint(f0) >> 16;
    d1 = __float_as_uint(f1) >> 16;
    d2 = __float_as_uint(f2) >> 16;
    d3 = __float_as_uint(f3) >> 16;
}

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(TC_LBO >> 4) << 16) | ((uint64_t)(TC_SBO >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor: fp32 accumulator, bf16 A and B, both K-major, N, M
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// Bounded wait on an mbarrier phase.  Every barrier here completes through this
// CTA's own tcgen05.commit, so a wait that gives up means the tensor cores have
// stalled: the caller then stops issuing work, skips every read of the
// accumulators and every result write, and reports the stall in the error word.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
    return done != 0;
}

// Matrix digits of V (rows x n used, [prime][n][n] normal form) in the operand
// layout: out[((prime * ct + c) * kc + k) * TC_VTILE_WORDS ...], digit planes of
// 64 rows x 32 K, zero outside rows x n.
__global__ void k_vinv_tc(const uint32_t *vinv, int n, int rows, int K, int nct, int nkc, uint16_t *out) {
    const int64_t per_prime = (int64_t)nct * nkc * TC_N * TC_KC;
    const int64_t total = per_prime * K;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / per_prime);
        int64_t rem = e % per_prime;
        const int c = (int)(rem / ((int64_t)nkc * TC_N * TC_KC));
        rem %= (int64_t)nkc * TC_N * TC_KC;
        const int k = (int)(rem / (TC_N * TC_KC));
        const int w = (int)(rem % (TC_N * TC_KC));
        const int rl = w / TC_KC, kl = w % TC_KC;
        const int r = c * TC_N + rl, j = k * TC_KC + kl;
        const uint32_t x = (r < rows && j < n) ? vinv[((int64_t)i * n + r) * n + j] : 0u;
        uint32_t d[4];
        tc_digits(x, d[0], d[1], d[2], d[3]);
        uint16_t *tile = out + (((int64_t)i * nct + c) * nkc + k) * (4 * TC_N * TC_KC);
        for (int t = 0; t < 4; ++t) tile[t * TC_N * TC_KC + tc_elem(rl, kl)] = (uint16_t)d[t];
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_interp_tc(ResLaunch L, const char *planblk, const GemmGroup *groups,
                                                     const GemmTile *tiles) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t bar[3];   // stage 0, stage 1 released; all MMAs done
    __shared__ uint32_t tmem_slot;
    __shared__ int64_t vbs[TC_M];              // value base of each row's pair (-1: none)
    if (stage_skipped(L)) return;                // whole CTA, before any tensor memory is taken
    const GemmTile T = tiles[blockIdx.x];
    const GemmGroup Gr = groups[T.group];
    const int n = Gr.n, rows = Gr.rows, mode = Gr.mode, i = T.prime;
    const int nkc = (n + TC_KC - 1) / TC_KC, nct = (n + TC_N - 1) / TC_N;   // tiles cover all n rows
    const int tid = threadIdx.x, warp = tid >> 5;
    const ModP M = L.mods[i];
    // this thread's pair (tensor-memory lane row = tid mod 128); the threads
    // tid + 128 t share the row and split its K groups and its columns
    const int row = tid & (TC_M - 1), part = tid >> 7;
    const int32_t *gpairs = (const int32_t *)(planblk + Gr.pairs_off);
    int64_t vb = -1, cb = 0;
    if (T.q0 + row < Gr.npairs) {
        const PairPlan &pp = L.plan[gpairs[T.q0 + row]];
        if (i < pp.k) {
            vb = pp.val_off + (int64_t)i * pp.Pe;
            cb = pp.cf_off + (int64_t)i * pp.P;
        }
    }
    if (part == 0) vbs[row] = vb;
    // resident operand (tile c0 < 0): the operand's digits for all of K stay in
    // shared memory (one slot per chunk) and the CTA runs every row tile of the
    // matrix against them; otherwise one row tile, operand and matrix streamed
    // through two stages
    const bool resident = T.c0 < 0;
    const int nrt = resident ? (rows + TC_N - 1) / TC_N : 1, ct0 = resident ? 0 : T.c0 / TC_N;
    const int xslots = resident ? nkc : 2, steps = nrt * nkc;
    unsigned char *xsm = tsm;                                        // X digit planes, per slot
    unsigned char *vsm = tsm + (size_t)xslots * TC_XSLOT;            // V digit planes, two stages
    uint32_t *raw = reinterpret_cast<uint32_t *>(vsm + 2 * TC_VSLOT);   // TC_M x 33 words
    const uint32_t *vt = (const uint32_t *)Gr.vtc + ((int64_t)i * nct + ct0) * nkc * TC_VTILE_WORDS;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bar[b])),
                         "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_slot;
    const uint32_t xbase = (uint32_t)__cvta_generic_to_shared(xsm), vbase = (uint32_t)__cvta_generic_to_shared(vsm);
    bool stalled = false;   // CTA-uniform: a wait gave up, no further MMA is issued
    bool acc_pending = false;   // a commit of the accumulators is issued and not yet seen complete
    int acc_phase = 0;          // completions of bar[2] seen (one per row tile)
    // software pipeline over steps (row tile, chunk): the loads of step st + 1
    // (operand rows: TC_M / TC_WARPS per warp, lanes along K, only while the operand
    // is still being staged; the 16 KB matrix block) are in flight while step st is
    // split into digits and multiplied, and during a row tile's epilogue
    const int lane = tid & 31;
    const uint32_t iota = mode >= GEMM_Q0 ? iota_mont(L, i) : 0u;
    uint32_t ra[TC_M / TC_WARPS][4];
    uint4 rv[4 * TC_VPLANE / 16 / TC_THREADS];
    auto preload = [&](int st) {
        const int c = st / nkc, kc = st - c * nkc;
        if (!resident || c == 0) {
            const int j = kc * TC_KC + lane;
#pragma unroll
            for (int it = 0; it < TC_M / TC_WARPS; ++it) {
                const int64_t b = vbs[warp + TC_WARPS * it];
                if (b >= 0 && j < n) operand_loads(L.val + b, mode, j, n, ra[it]);
                else ra[it][0] = ra[it][1] = ra[it][2] = ra[it][3] = 0u;
            }
        }
        const uint4 *src = reinterpret_cast<const uint4 *>(vt + ((int64_t)c * nkc + kc) * TC_VTILE_WORDS);
#pragma unroll
        for (int u = 0; u < 4 * TC_VPLANE / 16 / TC_THREADS; ++u) rv[u] = __ldg(src + tid + TC_THREADS * u);
    };
    const int ostride = gemm_ostride(mode), ooff = gemm_ooff(mode);
    const uint64_t off_lo = (uint64_t)M.p << 20, off_hi = (uint64_t)M.p << 11;
    // epilogue of row tile ct: lane tid holds pair q0 + tid; combine the diagonals
    // per coefficient
    auto epilogue = [&](int ct) {
        for (int c0 = part * TC_CPT; c0 < (part + 1) * TC_CPT; c0 += 4) {
            uint32_t v[TC_DIAG][4];
#pragma unroll
            for (int u = 0; u < TC_DIAG; ++u) {
                const uint32_t addr = tbase + ((uint32_t)((warp & 3) * 32) << 16) + u * TC_N + c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v[u][0]), "=r"(v[u][1]), "=r"(v[u][2]), "=r"(v[u][3])
                             : "r"(addr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (vb < 0) continue;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = ct * TC_N + c0 + e;
                if (r >= rows) break;
                int64_t d[TC_DIAG];
#pragma unroll
                for (int u = 0; u < TC_DIAG; ++u) d[u] = (int64_t)__float2int_rn(__uint_as_float(v[u][e]));
                // C = hi 2^32 + lo with |lo| < 2^49, |hi| < 2^41; both made positive by
                // multiples of p, then coef = hi + lo R^-1 (mod p)
                const int64_t lo = d[0] + (d[1] << 8) + (d[2] << 16) + (d[3] << 24);
                const int64_t hi = d[4] + (d[5] << 8) + (d[6] << 16);
                const uint64_t tl = (uint64_t)lo + off_lo, th = (uint64_t)hi + off_hi;
                const uint32_t rl = mp_redc((uint32_t)tl, (uint32_t)(tl >> 32), M.p, M.pinv);
                const uint32_t rh = mp_mul(mp_redc((uint32_t)th, (uint32_t)(th >> 32), M.p, M.pinv), M.r2, M);
                L.cf[cb + (int64_t)r * ostride + ooff] = mp_add(rh, rl, M.p);
            }
        }
    };
    preload(0);
    for (int st = 0; st < steps; ++st) {
        const int c = st / nkc, kc = st - c * nkc, s = st & 1;
        const bool stage_x = !resident || c == 0;
        const int xs_slot = resident ? kc : s;
        // stage s (and the streamed operand slot s) is free once the MMAs of step
        // st - 2 have read it
        const bool late = st >= 2 && !tc_wait((uint32_t)__cvta_generic_to_shared(&bar[s]), ((st >> 1) - 1) & 1);
        // the loaded chunk's operand (formed from its values, below p) into raw rows
        // (pitch 33 words, not read by the tensor cores)
        if (stage_x) {
#pragma unroll
            for (int it = 0; it < TC_M / TC_WARPS; ++it)
                raw[(warp + TC_WARPS * it) * 33 + lane] = operand_combine(ra[it], mode, iota, M);
        }
        // a wait that gave up on any thread ends the loop on all of them before
        // anything is written into a stage an MMA may still be reading
        if (__syncthreads_or(late)) {
            stalled = true;
            break;
        }
        {
            uint4 *dst = reinterpret_cast<uint4 *>(vsm + (size_t)s * TC_VSLOT);
#pragma unroll
            for (int u = 0; u < 4 * TC_VPLANE / 16 / TC_THREADS; ++u) dst[tid + TC_THREADS * u] = rv[u];
        }
        if (st + 1 < steps) preload(st + 1);
        // each thread splits TC_KG K groups of its row into four digit planes
        if (stage_x) {
            unsigned char *xd = xsm + (size_t)xs_slot * TC_XSLOT;
            uint32_t pk[4][TC_KG][4];   // [digit][k-group][word]: two bf16 per word
#pragma unroll
            for (int g = 0; g < TC_KG; ++g)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int kk = (TC_KG * part + g) * 8 + h * 2;
                    uint32_t dlo[4], dhi[4];
                    tc_digits(raw[row * 33 + kk], dlo[0], dlo[1], dlo[2], dlo[3]);
                    tc_digits(raw[row * 33 + kk + 1], dhi[0], dhi[1], dhi[2], dhi[3]);
#pragma unroll
                    for (int t = 0; t < 4; ++t) pk[t][g][h] = dlo[t] | (dhi[t] << 16);
                }
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int g = 0; g < TC_KG; ++g)
                    *reinterpret_cast<uint4 *>(xd + t * TC_XPLANE + 2 * tc_elem(row, (TC_KG * part + g) * 8)) =
                        make_uint4(pk[t][g][0], pk[t][g][1], pk[t][g][2], pk[t][g][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        const bool last = kc == nkc - 1;   // row tile c complete after this step
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t xs = xbase + xs_slot * TC_XSLOT, vs = vbase + s * TC_VSLOT;
#pragma unroll
            for (int ks = 0; ks < TC_KC / 16; ++ks)
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int u = a + b;
                        const uint32_t acc = (kc > 0 || ks > 0 || a != (u > 3 ? u - 3 : 0)) ? 1u : 0u;
                        const uint64_t da = tc_sdesc(xs + a * TC_XPLANE + ks * 2 * TC_LBO);
                        const uint64_t db = tc_sdesc(vs + b * TC_VPLANE + ks * 2 * TC_LBO);
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tbase + u * TC_N),
                            "l"(da), "l"(db), "r"(tc_idesc()), "r"(acc));
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                (uint32_t)__cvta_generic_to_shared(&bar[s])));
            // the accumulators of the row tile are complete when every MMA so far is
            if (last)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    (uint32_t)__cvta_generic_to_shared(&bar[2])));
        }
        if (last) {
            acc_pending = true;
            if (!__syncthreads_and(tc_wait((uint32_t)__cvta_generic_to_shared(&bar[2]), acc_phase & 1))) {
                stalled = true;
                break;
            }
            acc_pending = false;
            ++acc_phase;
            asm volatile("tcgen05.fence::after_thread_sync;");
            epilogue(ct0 + c);
            // every read of the accumulators is done before the next row tile's
            // first MMA overwrites them
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
    }
    if (stalled) {
        // one more commit tracks every MMA issued, unless the row tile's own commit
        // is still outstanding; nothing is read or written, the tensor memory is
        // given back only when they have completed (or that wait gives up too)
        if (tid == 0 && !acc_pending)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                (uint32_t)__cvta_generic_to_shared(&bar[2])));
        __syncthreads_and(tc_wait((uint32_t)__cvta_generic_to_shared(&bar[2]), acc_phase & 1));
        if (tid == 0) atomicExch(L.err, kErrTensorStall);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

// digit tiles of a cached matrix: K primes x ceil(rows/64) x ceil(n/32) blocks of 16 KB
size_t vinv_tc_bytes(int n, int rows, int K) {
    return (size_t)K * ((rows + TC_N - 1) / TC_N) * ((n + TC_KC - 1) / TC_KC) * (4 * TC_VPLANE);
}

cudaError_t launch_vinv_tc(const uint32_t *vinv, int n, int rows, int K, uint16_t *out, cudaStream_t s) {
    const int nct = (rows + TC_N - 1) / TC_N, nkc = (n + TC_KC - 1) / TC_KC;
    const int64_t total = (int64_t)K * nct * nkc * TC_N * TC_KC;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_vinv_tc<<<grid, 256, 0, s>>>(vinv, n, rows, K, nct, nkc, out);
    return cudaGetLastError();
}

// One CTA per tile (q0 a multiple of 128; c0 a multiple of 64, or -1 for every row
// tile on a resident operand of at most kTcResidentChunks chunks).  The shared
// memory request (operand slots, two matrix stages, the raw rows; at least past half
// the SM) keeps one CTA per SM, which also owns the SM's 512 tensor-memory columns.
constexpr size_t kTcSmemMax = (size_t)kTcResidentChunks * TC_XSLOT + 2 * TC_VSLOT + TC_RAW;
static_assert(kTcSmemMax <= 227 * 1024, "the resident operand fits one CTA's shared memory");

cudaError_t launch_interp_tc(const ResLaunch &L, const char *planblk, const GemmGroup *groups, const GemmTile *tiles,
                             int ntiles, int xslots, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (xslots < 2 || xslots > kTcResidentChunks) return cudaErrorInvalidValue;
    const size_t smem = std::max<size_t>((size_t)xslots * TC_XSLOT + 2 * TC_VSLOT + TC_RAW, (size_t)120 * 1024);
    k_interp_tc<<<ntiles, TC_THREADS, smem, s>>>(L, planblk, groups, tiles);
    return cudaGetLastError();
}

cudaError_t configure_interp_tc_kernel() {
    return cudaFuncSetAttribute(k_interp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
}

}  // namespace gbr
