// Square-free factorisation R = u * prod_i r_i^i of integer polynomials
// (Section 2.1, Projection Phase: the square-free, pairwise coprime factors r_i
// of R = res(f, f_y, y), by Yun's algorithm), multi-modular like the rest of the
// path:
//   reduce   every coefficient of R modulo a run of table primes (device)
//   yun      one warp per (polynomial, prime): Yun's algorithm over F_p -
//            G = gcd(A, A'), C = A / G, D = A' / G - C', then r_i = gcd(C, D),
//            C = C / r_i, D = D / r_i - C' until deg C = 0 (A = R / lc(R), p > deg R)
//   (host)   the primes whose square-free part has the largest degree all share
//            the true degree pattern (a prime that merges factors lowers it)
//   lift     Garner lift of lc(R) * (monic r_i mod p): that is (lc R / lc r_i) r_i,
//            whose 1-norm is at most 2^deg(r_i) ||R||_2 (Mignotte, since r_i | R)
//   (host)   primitive parts (big-integer gcds), u = lc(R) / prod lc(r_i)^i
//   verify   R = u prod r_i^i modulo primes whose product exceeds twice both
//            sides' coefficient bounds, so the identity holds over Z (device).
// A failed check (too few lucky primes among those tried) doubles the primes.
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <thread>

#include "gbr_bigint.h"
#include "gbr_core.h"
#include "gbr_sqf_host.h"

namespace gbr {

struct SqfJob {
    int32_t n, limbs;      // degree of R, 32-bit limbs per coefficient
    int64_t mag_off;       // R's limbs in the limb buffer (words)
    int64_t sign_off;      // R's signs (bytes)
    int64_t res_off;       // residues [slot][n + 1]
    int64_t out_off;       // monic factors mod p, normal form, packed: [slot][2n + 2]
    int64_t pat_off;       // [slot][n + 2] int32: m (-1: prime unusable), deg r_1..r_m
    int64_t lsel_off;      // lifted primes: int32 slot indices, lift_k of them
    int64_t gtab_off;      // Garner table of the lifted primes
    int64_t lift_off;      // lifted coefficients [coef][lift_L] limbs
    int64_t lsign_off;     // and their signs
    int64_t ver_off;       // candidate factors for the check: limbs [coef][ver_L], signs after
    int32_t lift_k, lift_L, ver_L, nfac;
    int32_t status, pad;
    int64_t red0, lift0;   // first item of this job in the reduce and lift grids
};

// the job whose item range [start, next start) holds item (starts ascending)
template <int64_t SqfJob::*F>
__device__ int sqf_find(const SqfJob *jobs, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].*F <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct SqfLaunch {
    const SqfJob *jobs;
    int32_t njobs, p0, nprimes;   // table primes p0 .. p0 + nprimes - 1 (one slot each)
    const ModP *mods;
    const uint32_t *limbs;
    const int8_t *signs;
    uint32_t *res;
    uint32_t *out;
    int32_t *pat;
    const int32_t *lsel;
    uint32_t *gtab;
    uint32_t *lift;
    int8_t *lsign;
    const uint32_t *ver;          // candidate factors' limbs; each job's u first, then r_1..r_m
    const int32_t *ver_deg;       // per job: degrees of r_1..r_m at ver_deg + job * (max_fac + 1)
    int32_t *ver_fail;
    int32_t *err;
    int32_t max_fac;
};

// ------------------------------------------------------------------ reduce

// residue slot s of job j, coefficient c: Horner over the limbs from the top,
// acc = (acc * 2^32 + limb) R: with acc kept as V R, (acc + limb mod p) R^2 R^-1
__global__ void k_sqf_reduce(SqfLaunch L, int64_t total) {
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
        const int j = sqf_find<&SqfJob::red0>(L.jobs, L.njobs, it);
        const SqfJob &J = L.jobs[j];
        const int64_t rem = it - J.red0;
        const int s = (int)(rem / (J.n + 1)), c = (int)(rem % (J.n + 1));
        const ModP M = L.mods[L.p0 + s];
        const uint32_t *x = L.limbs + J.mag_off + (int64_t)c * J.limbs;
        uint32_t acc = 0u;
        for (int l = J.limbs - 1; l >= 0; --l) {
            uint32_t v = x[l];
            v = v >= 2u * M.p ? v - 2u * M.p : v;
            v = v >= M.p ? v - M.p : v;
            acc = mp_mul(mp_add(acc, v, M.p), M.r2, M);
        }
        if (L.signs[J.sign_off + c] < 0) acc = mp_neg(acc, M.p);
        L.res[J.res_off + (int64_t)s * (J.n + 1) + c] = acc;
    }
}

// ------------------------------------------------------------------ Yun over F_p, one warp

__device__ __forceinline__ int wp_degree(const uint32_t *a, int d) {
    while (d >= 0 && a[d] == 0u) --d;
    return d;
}

// monic gcd of X (degree dx) and Y (degree dy), both destroyed; returns the
// buffer holding it and its degree in *dg (-1 when both are zero)
__device__ uint32_t *wp_gcd(uint32_t *X, int dx, uint32_t *Y, int dy, int *dg, const ModP &M, int lane) {
    dx = wp_degree(X, dx);
    dy = wp_degree(Y, dy);
    while (dy >= 0) {
        if (dx < dy) {
            uint32_t *t = X; X = Y; Y = t;
            int ti = dx; dx = dy; dy = ti;
            continue;
        }
        const uint32_t zeta = Y[dy], q = X[dx];
        const int s = dx - dy;
        for (int t = lane; t < dx; t += 32)
            X[t] = t >= s ? mp_mulsub(zeta, X[t], q, Y[t - s], M) : mp_mul(zeta, X[t], M);
        __syncwarp();
        dx = wp_degree(X, dx - 1);
    }
    *dg = dx;
    if (dx >= 0) {
        const uint32_t il = mp_inv(X[dx], M);
        __syncwarp();
        for (int t = lane; t <= dx; t += 32) X[t] = mp_mul(X[t], il, M);
        __syncwarp();
    }
    return X;
}

// Q = N / V for a monic V of degree dv dividing N (degree dn); N is destroyed
__device__ void wp_div(uint32_t *N, int dn, const uint32_t *V, int dv, uint32_t *Q, const ModP &M, int lane) {
    for (int k = dn; k >= dv; --k) {
        const uint32_t q = N[k];
        __syncwarp();
        if (lane == 0) Q[k - dv] = q;
        for (int t = lane; t < dv; t += 32) N[k - dv + t] = mp_sub(N[k - dv + t], mp_mul(q, V[t], M), M.p);
        __syncwarp();
    }
}

// D <- D - C' (C of degree dc, D of degree at most dc - 1 beforehand)
__device__ void wp_sub_deriv(uint32_t *D, int dd, const uint32_t *C, int dc, const ModP &M, int lane) {
    for (int t = lane; t < dc; t += 32) {
        const uint32_t dv = mp_mul(C[t + 1], mp_to((uint32_t)(t + 1), M), M);
        D[t] = mp_sub(t <= dd ? D[t] : 0u, dv, M.p);
    }
    __syncwarp();
}

__global__ void k_sqf_yun(SqfLaunch L, int stride) {
    extern __shared__ uint32_t sm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t *buf[6];
    for (int b = 0; b < 6; ++b) buf[b] = sm + (size_t)(wid * 6 + b) * stride;
    int64_t total = (int64_t)L.njobs * L.nprimes;
    for (int64_t it = (int64_t)blockIdx.x * nw + wid; it < total; it += (int64_t)gridDim.x * nw) {
        const int j = (int)(it / L.nprimes), s = (int)(it % L.nprimes);
        const SqfJob &J = L.jobs[j];
        const int n = J.n;
        const ModP M = L.mods[L.p0 + s];
        int32_t *pat = L.pat + J.pat_off + (int64_t)s * (n + 2);
        uint32_t *out = L.out + J.out_off + (int64_t)s * (2 * n + 2);
        const uint32_t *A0 = L.res + J.res_off + (int64_t)s * (n + 1);
        uint32_t *A = buf[0], *B = buf[1];
        for (int t = lane; t <= n; t += 32) A[t] = A0[t];
        __syncwarp();
        if (A[n] == 0u) {   // p divides lc(R): not usable
            if (lane == 0) pat[0] = -1;
            continue;
        }
        const uint32_t il = mp_inv(A[n], M);
        __syncwarp();
        for (int t = lane; t <= n; t += 32) A[t] = mp_mul(A[t], il, M);
        __syncwarp();
        for (int t = lane; t < n; t += 32) B[t] = mp_mul(A[t + 1], mp_to((uint32_t)(t + 1), M), M);
        __syncwarp();
        // G = gcd(A, A') on copies
        uint32_t *X = buf[2], *Y = buf[3];
        for (int t = lane; t <= n; t += 32) {
            X[t] = A[t];
            Y[t] = t < n ? B[t] : 0u;
        }
        __syncwarp();
        int dg;
        uint32_t *G = wp_gcd(X, n, Y, n - 1, &dg, M, lane);
        uint32_t *C = buf[4], *D = buf[5];
        wp_div(A, n, G, dg, C, M, lane);
        int dc = n - dg;
        wp_div(B, n - 1, G, dg, D, M, lane);
        int dd = n - 1 - dg;
        wp_sub_deriv(D, dd, C, dc, M, lane);
        dd = wp_degree(D, dc - 1);
        int m = 0, off = 0;
        bool bad = false;
        int ic = 4, id = 5;   // buffers holding C and D
        while (dc > 0) {
            // r = gcd(C, D) on copies in two free buffers; the quotients go to the other two
            int fr[4], nf = 0;
            for (int b = 0; b < 6; ++b)
                if (b != ic && b != id) fr[nf++] = b;
            uint32_t *F0 = buf[fr[0]], *F1 = buf[fr[1]], *N0 = buf[fr[2]], *N1 = buf[fr[3]];
            for (int t = lane; t <= dc; t += 32) {
                F0[t] = C[t];
                F1[t] = t <= dd ? D[t] : 0u;
            }
            __syncwarp();
            int dr;
            uint32_t *Rf = wp_gcd(F0, dc, F1, dd, &dr, M, lane);
            if (dr < 0 || off + dr + 1 > 2 * n + 2 || m >= n + 1) {
                bad = true;
                break;
            }
            for (int t = lane; t <= dr; t += 32) out[off + t] = mp_from(Rf[t], M);
            if (lane == 0) pat[1 + m] = dr;
            off += dr + 1;
            ++m;
            // C <- C / r, D <- D / r - C'
            wp_div(C, dc, Rf, dr, N0, M, lane);
            const int ndc = dc - dr;
            if (dd >= 0) wp_div(D, dd, Rf, dr, N1, M, lane);
            int ndd = dd >= 0 ? dd - dr : -1;
            for (int t = lane; t < ndc; t += 32)
                if (t > ndd) N1[t] = 0u;
            __syncwarp();
            wp_sub_deriv(N1, ndd, N0, ndc, M, lane);
            C = N0;
            D = N1;
            ic = fr[2];
            id = fr[3];
            dc = ndc;
            dd = wp_degree(D, dc - 1);
        }
        __syncwarp();
        if (lane == 0) pat[0] = bad ? -1 : m;
        __syncwarp();
    }
}

// ------------------------------------------------------------------ lift

// Garner constants of each job's lifted primes: tab[i] = (prod_{j<i} p_j)^-1 mod
// p_i, then p_j mod p_i (Montgomery) for j < i
__global__ void k_sqf_garner(SqfLaunch L) {
    for (int j = blockIdx.x; j < L.njobs; j += gridDim.x) {
        const SqfJob &J = L.jobs[j];
        if (J.status != 0 || J.lift_k <= 0) continue;
        const int32_t *sel = L.lsel + J.lsel_off;
        uint32_t *tab = L.gtab + J.gtab_off;
        for (int i = threadIdx.x; i < J.lift_k; i += blockDim.x) {
            const ModP M = L.mods[L.p0 + sel[i]];
            uint32_t prod = M.r1;
            uint32_t *pm = tab + J.lift_k + (int64_t)i * (i - 1) / 2;
            for (int q = 0; q < i; ++q) {
                uint32_t pq = L.mods[L.p0 + sel[q]].p;
                pq = pq >= M.p ? pq - M.p : pq;
                pm[q] = mp_to(pq, M);
                prod = mp_mul(prod, pm[q], M);
            }
            tab[i] = mp_inv(prod, M);
        }
    }
}

// one thread per (job, packed factor coefficient): v_i = lc(R) * coefficient mod
// p_i over the lifted primes, Garner digits in shared memory, symmetric lift
__global__ void k_sqf_lift(SqfLaunch L, int KM, int LM, int64_t total) {
    extern __shared__ uint32_t sm[];
    const int BS = blockDim.x;
    uint32_t *v = sm + threadIdx.x;
    uint32_t *limb = sm + (size_t)KM * BS + threadIdx.x;
    for (int64_t it = blockIdx.x * (int64_t)BS + threadIdx.x; it < total; it += (int64_t)gridDim.x * BS) {
        const int j = sqf_find<&SqfJob::lift0>(L.jobs, L.njobs, it);
        const SqfJob &J = L.jobs[j];
        if (J.status != 0 || it - J.lift0 >= J.nfac) continue;
        const int e = (int)(it - J.lift0), k = J.lift_k;
        const int32_t *sel = L.lsel + J.lsel_off;
        const uint32_t *tab = L.gtab + J.gtab_off;
        for (int i = 0; i < k; ++i) {
            const int s = sel[i];
            const ModP M = L.mods[L.p0 + s];
            const uint32_t lc = L.res[J.res_off + (int64_t)s * (J.n + 1) + J.n];   // Montgomery
            const uint32_t c = L.out[J.out_off + (int64_t)s * (2 * J.n + 2) + e];  // normal
            v[i * BS] = mp_mul(lc, c, M);                                          // lc * c, normal
        }
        for (int i = 1; i < k; ++i) {
            const ModP M = L.mods[L.p0 + sel[i]];
            const uint32_t *pmi = tab + k + (int64_t)i * (i - 1) / 2;
            uint32_t t = v[(i - 1) * BS];
            t = t >= M.p ? t - M.p : t;
            for (int q = i - 2; q >= 0; --q) {
                uint32_t vq = v[q * BS];
                vq = vq >= M.p ? vq - M.p : vq;
                t = mp_add(mp_mul(t, pmi[q], M), vq, M.p);
            }
            v[i * BS] = mp_mul(mp_sub(v[i * BS], t, M.p), tab[i], M);
        }
        int cmp = 0;
        for (int i = k - 1; i >= 0 && cmp == 0; --i) {
            const uint32_t d = v[i * BS], h = (L.mods[L.p0 + sel[i]].p - 1u) >> 1;
            cmp = (d > h) - (d < h);
        }
        const bool neg = cmp > 0;
        int nl = 0;
        for (int i = k - 1; i >= 0; --i) {
            const uint32_t p = L.mods[L.p0 + sel[i]].p;
            uint32_t d = v[i * BS];
            if (neg) d = p - 1u - d;
            uint32_t carry = d;
            for (int l = 0; l < nl; ++l) {
                const uint64_t t = (uint64_t)limb[l * BS] * p + carry;
                limb[l * BS] = (uint32_t)t;
                carry = (uint32_t)(t >> 32);
            }
            if (carry && nl < LM) limb[(nl++) * BS] = carry;
        }
        if (neg) {
            int l = 0;
            for (; l < nl; ++l)
                if (++limb[l * BS] != 0u) break;
            if (l == nl && nl < LM) limb[(nl++) * BS] = 1u;
        }
        if (nl > J.lift_L) atomicExch(L.err, 7);
        uint32_t *o = L.lift + J.lift_off + (int64_t)e * J.lift_L;
        for (int l = 0; l < J.lift_L; ++l) o[l] = l < nl ? limb[l * BS] : 0u;
        L.lsign[J.lsign_off + e] = nl == 0 ? 0 : (neg ? -1 : 1);
    }
}

// ------------------------------------------------------------------ verify

// one warp per (job, prime): u * prod r_i^i mod p against R mod p; the candidate
// factors come as limbs + signs (u first, then r_1..r_m, each coefficient ver_L
// limbs); reductions as in k_sqf_reduce
__device__ uint32_t wp_reduce_limbs(const uint32_t *x, int nl, int sign, const ModP &M) {
    uint32_t acc = 0u;
    for (int l = nl - 1; l >= 0; --l) {
        uint32_t v = x[l];
        v = v >= 2u * M.p ? v - 2u * M.p : v;
        v = v >= M.p ? v - M.p : v;
        acc = mp_mul(mp_add(acc, v, M.p), M.r2, M);
    }
    return sign < 0 ? mp_neg(acc, M.p) : acc;
}

__global__ void k_sqf_verify(SqfLaunch L, int stride) {
    extern __shared__ uint32_t sm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t *P = sm + (size_t)wid * 3 * stride, *Fb = P + stride, *T = Fb + stride;
    int64_t total = (int64_t)L.njobs * L.nprimes;
    for (int64_t it = (int64_t)blockIdx.x * nw + wid; it < total; it += (int64_t)gridDim.x * nw) {
        const int j = (int)(it / L.nprimes), s = (int)(it % L.nprimes);
        const SqfJob &J = L.jobs[j];
        if (J.status != 0) continue;
        const ModP M = L.mods[L.p0 + s];
        const int n = J.n, VL = J.ver_L;
        const uint32_t *vb = L.ver + J.ver_off;
        // number of coefficients stored before the signs: u (1) + sum (deg r_i + 1)
        const int32_t *degs = L.ver_deg + (int64_t)j * (L.max_fac + 1);
        int ncoef = 1;
        for (int i = 0; i < J.nfac; ++i) ncoef += degs[i] + 1;
        const int8_t *sg = reinterpret_cast<const int8_t *>(vb + (int64_t)ncoef * VL);
        // P = u
        if (lane == 0) P[0] = wp_reduce_limbs(vb, VL, sg[0], M);
        int dp = 0;
        int cur = 1;
        __syncwarp();
        for (int i = 0; i < J.nfac; ++i) {
            const int df = degs[i];
            for (int t = lane; t <= df; t += 32)
                Fb[t] = wp_reduce_limbs(vb + (int64_t)(cur + t) * VL, VL, sg[cur + t], M);
            __syncwarp();
            for (int e = 0; e <= i; ++e) {   // multiply i + 1 times (factor of multiplicity i + 1)
                if (dp + df > n) break;
                for (int t = lane; t <= dp + df; t += 32) {
                    uint32_t acc = 0u;
                    const int a0 = t - df > 0 ? t - df : 0, a1 = t < dp ? t : dp;
                    for (int a = a0; a <= a1; ++a) acc = mp_add(acc, mp_mul(P[a], Fb[t - a], M), M.p);
                    T[t] = acc;
                }
                __syncwarp();
                dp += df;
                for (int t = lane; t <= dp; t += 32) P[t] = T[t];
                __syncwarp();
            }
            cur += df + 1;
        }
        // compare with R mod p (both Montgomery)
        const uint32_t *R = L.res + J.res_off + (int64_t)s * (n + 1);
        bool ok = dp == n;
        for (int t = lane; t <= n && ok; t += 32) ok = ok && P[t] == R[t];
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) atomicExch(L.ver_fail + j, 1);
        __syncwarp();
    }
}

}  // namespace gbr

// ------------------------------------------------------------------ host driver

using namespace gbr;
using namespace gbr::sqfh;

namespace {

struct SqfHost {
    int n = -1;                        // degree of R (-1: zero)
    bn::Big lc;                        // leading coefficient of R
    double l2norm2 = 0.0, l2inf = 0.0; // log2 ||R||_2, log2 ||R||_inf
    int status = 0;                    // 0 pending, 1 done
    std::vector<int> pat;              // chosen degree pattern
    std::vector<int> lucky;            // slots with that pattern
    bn::Big u;
    std::vector<FlatPoly> fac;         // r_1..r_m
};

struct DevBufs {
    gbr_ctx *c;
    std::vector<void *> v;
    void *get(size_t b) {
        void *x = c->dalloc(b ? b : 16);
        if (x) v.push_back(x);
        return x;
    }
    ~DevBufs() {
        for (void *x : v) c->dfree(x);
    }
};

int sqf_blocks(const void *k, int block, size_t smem, int64_t need) {
    int per_sm = 0, dev = 0, sms = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = (int64_t)std::max(per_sm, 1) * sms;
    return (int)std::max<int64_t>(1, std::min<int64_t>(cap, need));
}

// warps per block for the shared-memory polynomial kernels: `bufs` buffers of
// `stride` words per warp within kMaxDynSmem
int sqf_warps(int bufs, int stride) {
    const size_t per = (size_t)bufs * stride * 4;
    int w = (int)std::min<size_t>(4, kMaxDynSmem / per);
    return std::max(w, 0);
}



}  // namespace

// inputs whose lift would take at least this many primes get the two-prime
// square-free test first
constexpr int kSqfTestMinPrimes = 12;

// copies of the square-free path, counted for gbr_stats like the gcd path's
static cudaError_t sqf_copy(gbr_ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                            cudaStream_t s) {
    if (kind == cudaMemcpyHostToDevice) c->gcd_h2d += (int64_t)bytes;
    else c->gcd_d2h += (int64_t)bytes;
    return cudaMemcpyAsync(dst, src, bytes, kind, s);
}

// The modular stage: R modulo the first K table primes and Yun's algorithm over
// each, for the jobs `pend`; fills the job table, the launch parameters (residues
// and monic factors stay on the device) and the degree patterns on the host.
struct SqfStage {
    std::vector<SqfJob> J;
    std::vector<int32_t> pat;
    SqfLaunch L{};
    SqfJob *d_jobs = nullptr;
    int stride = 0;
};

static int sqf_modular_stage(gbr_ctx *c, DevBufs &B, const std::vector<int> &pend, const std::vector<SqfHost> &H,
                             const gbr_bigpoly *in, const std::vector<int64_t> &mag_off,
                             const std::vector<int64_t> &sign_off, const uint32_t *d_limbs, const int8_t *d_signs,
                             int K, SqfStage &st) {
    cudaStream_t s = c->stream;
    const int nj = (int)pend.size();
    std::vector<SqfJob> &J = st.J;
    J.assign(nj, SqfJob{});
    int64_t res_w = 0, out_w = 0, pat_w = 0, red = 0;
    int maxn = 0;
    for (int q = 0; q < nj; ++q) {
        const int j = pend[q];
        SqfJob &x = J[q];
        std::memset(&x, 0, sizeof(x));
        x.n = H[j].n;
        x.limbs = in[j].limbs;
        x.mag_off = mag_off[j];
        x.sign_off = sign_off[j];
        x.res_off = res_w;
        x.out_off = out_w;
        x.pat_off = pat_w;
        x.red0 = red;
        res_w += (int64_t)K * (x.n + 1);
        out_w += (int64_t)K * (2 * x.n + 2);
        pat_w += (int64_t)K * (x.n + 2);
        red += (int64_t)K * (x.n + 1);
        maxn = std::max(maxn, x.n);
    }
    const int stride = maxn + 2;
    const int nwy = sqf_warps(6, stride);
    if (nwy < 1) return c->fail(GBR_ELIMIT, "square-free input degree too large for shared memory");
    SqfJob *d_jobs = (SqfJob *)B.get(sizeof(SqfJob) * nj);
    uint32_t *d_res = (uint32_t *)B.get((size_t)res_w * 4);
    uint32_t *d_out = (uint32_t *)B.get((size_t)out_w * 4);
    int32_t *d_pat = (int32_t *)B.get((size_t)pat_w * 4);
    if (!d_jobs || !d_res || !d_out || !d_pat) return c->fail(GBR_ENOMEM, "device budget too small for the square-free stage");
    SqfLaunch &L = st.L;
    L = SqfLaunch{};
    L.jobs = d_jobs;
    L.njobs = nj;
    L.p0 = 0;
    L.nprimes = K;
    L.mods = c->d_mods;
    L.limbs = d_limbs;
    L.signs = d_signs;
    L.res = d_res;
    L.out = d_out;
    L.pat = d_pat;
    L.err = c->d_err;
    cudaError_t e = sqf_copy(c, d_jobs, J.data(), sizeof(SqfJob) * nj, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, 4, s);
    if (e == cudaSuccess) {
        k_sqf_reduce<<<sqf_blocks((const void *)k_sqf_reduce, 256, 0, (red + 255) / 256), 256, 0, s>>>(L, red);
        e = cudaGetLastError();
        ++c->gcd_kernels;
    }
    if (e == cudaSuccess) {
        const size_t smem = (size_t)nwy * 6 * stride * 4;
        k_sqf_yun<<<sqf_blocks((const void *)k_sqf_yun, nwy * 32, smem, ((int64_t)nj * K + nwy - 1) / nwy), nwy * 32,
                    smem, s>>>(L, stride);
        e = cudaGetLastError();
        ++c->gcd_kernels;
        c->gcd_subproblems += (int64_t)nj * K;
    }
    st.pat.resize(pat_w);
    if (e == cudaSuccess) e = sqf_copy(c, st.pat.data(), d_pat, (size_t)pat_w * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "square-free modular stage", e);
    st.d_jobs = d_jobs;
    st.stride = stride;
    return GBR_OK;
}

static int sqf_batch_locked(gbr_ctx *c, int n, const gbr_bigpoly *in, gbr_sqf *out) {
    cudaStream_t s = c->stream;
    const int NP = num_primes();
    const int threads = (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
    c->gcd_kernels = c->gcd_subproblems = c->gcd_h2d = c->gcd_d2h = 0;
    std::vector<SqfHost> H(n);
    // ---- host view of every input; constants and zero are finished here
    for (int j = 0; j < n; ++j) {
        const gbr_bigpoly &P = in[j];
        if (P.deg >= 0 && (!P.mag || !P.sign || P.limbs < 1)) return c->fail(GBR_EINVAL, "bad input polynomial");
        int d = P.deg;
        while (d > GBR_MAX_UDEG && P.sign[d] == 0) --d;
        if (d > GBR_MAX_UDEG) return c->fail(GBR_ELIMIT, "square-free input degree above GBR_MAX_UDEG");
    }
    gbr_parallel_for(n, threads, [&](int lo, int hi) {
        for (int j = lo; j < hi; ++j) {
            const gbr_bigpoly &P = in[j];
            int d = P.deg;
            while (d >= 0 && P.sign[d] == 0) --d;
            H[j].n = d;
            if (d < 1) {
                H[j].status = 1;
                if (d == 0) H[j].u = bn::from_limbs(P.mag, P.limbs, P.sign[0]);
                continue;
            }
            H[j].lc = bn::from_limbs(P.mag + (size_t)d * P.limbs, P.limbs, P.sign[d]);
            const Norms nr = log2_norms(d + 1, [&](int t, const uint32_t *&x, size_t &nl) {
                x = P.mag + (size_t)t * P.limbs;
                nl = P.sign[t] ? bn::top(x, (size_t)P.limbs) : 0;
            });
            H[j].l2norm2 = nr.l2;
            H[j].l2inf = nr.linf;
        }
    });
    int64_t words = 0, signs = 0;
    std::vector<int64_t> mag_off(n, 0), sign_off(n, 0);
    std::vector<int> pend;
    for (int j = 0; j < n; ++j) {
        if (H[j].status) continue;
        pend.push_back(j);
        mag_off[j] = words;
        sign_off[j] = signs;
        words += (int64_t)(H[j].n + 1) * in[j].limbs;
        signs += H[j].n + 1;
    }
    DevBufs B{c, {}};
    uint32_t *d_limbs = nullptr;
    int8_t *d_signs = nullptr;
    if (!pend.empty()) {
        uint32_t *hl = (uint32_t *)c->pinned((size_t)words * 4 + (size_t)signs + 64, 0);
        if (!hl) return c->fail(GBR_ENOMEM, "pinned host staging");
        int8_t *hs = (int8_t *)(hl + words);
        gbr_parallel_for((int)pend.size(), threads, [&](int lo, int hi) {
            for (int q = lo; q < hi; ++q) {
                const int j = pend[q];
                std::memcpy(hl + mag_off[j], in[j].mag, (size_t)(H[j].n + 1) * in[j].limbs * 4);
                std::memcpy(hs + sign_off[j], in[j].sign, (size_t)H[j].n + 1);
            }
        });
        d_limbs = (uint32_t *)B.get((size_t)words * 4 + (size_t)signs + 64);
        if (!d_limbs) return c->fail(GBR_ENOMEM, "device budget too small for the square-free inputs");
        d_signs = (int8_t *)(d_limbs + words);
        cudaError_t e = sqf_copy(c, d_limbs, hl, (size_t)words * 4 + (size_t)signs, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "square-free upload", e);
    }
    // ---- square-free test: Yun modulo two primes.  A prime not dividing lc(R) whose
    // modular square-free part has degree n proves R square-free over Z (a repeated
    // factor g^2 of R would stay one modulo p, with deg(g mod p) = deg g); then
    // R = u * pp(R) and nothing needs lifting.  Most projection resultants are
    // square-free, so this settles them with two primes instead of the lift's count;
    // it pays for itself once that count is large (kSqfTestMinPrimes and above).
    std::vector<int> tpend, rest;
    for (int j : pend)
        (primes_for_bits(H[j].n + H[j].l2norm2 + 3.0) + 4 >= kSqfTestMinPrimes ? tpend : rest).push_back(j);
    if (!tpend.empty()) {
        SqfStage ST;
        const int KA = 2;
        int rc = sqf_modular_stage(c, B, tpend, H, in, mag_off, sign_off, d_limbs, d_signs, KA, ST);
        if (rc) return rc;
        std::vector<char> done(tpend.size(), 0), fail(tpend.size(), 0);
        gbr_parallel_for((int)tpend.size(), threads, [&](int lo, int hi) {
            bn::Scratch S;
            for (int q = lo; q < hi; ++q) {
                const int j = tpend[q];
                SqfHost &h = H[j];
                const int32_t *pq = ST.pat.data() + ST.J[q].pat_off;
                bool sf = false;
                for (int sl = 0; sl < KA && !sf; ++sl) {
                    const int32_t *ps = pq + (int64_t)sl * (h.n + 2);
                    sf = ps[0] == 1 && ps[1] == h.n;
                }
                if (!sf) continue;
                h.fac.assign(1, FlatPoly());
                if (!primitive_part(in[j].mag, in[j].sign, h.n, in[j].limbs, h.fac[0], S) ||
                    !bn::divexact(h.lc, lead(h.fac[0]), h.u, S)) {
                    fail[q] = 1;
                    continue;
                }
                h.pat.assign(1, h.n);
                done[q] = 1;
            }
        });
        for (size_t q = 0; q < tpend.size(); ++q) {
            if (fail[q]) return c->fail(GBR_EDEVICE, "square-free: primitive part of a square-free input failed");
            if (done[q]) H[tpend[q]].status = 1;
            else rest.push_back(tpend[q]);
        }
        std::sort(rest.begin(), rest.end());
    }
    pend.swap(rest);
    // ---- attempts: K primes from the start of the table, doubled on failure
    int K = 0;
    for (int j : pend) K = std::max(K, primes_for_bits(H[j].n + H[j].l2norm2 + 3.0) + 4);
    if (K > NP) return c->fail(GBR_ELIMIT, "square-free input needs more than the table's primes");
    while (!pend.empty()) {
        if (K > NP) return c->fail(GBR_EVERIFY, "square-free check failed with every table prime");
        const int nj = (int)pend.size();
        SqfStage ST;
        int rc = sqf_modular_stage(c, B, pend, H, in, mag_off, sign_off, d_limbs, d_signs, K, ST);
        if (rc) return rc;
        std::vector<SqfJob> &J = ST.J;
        std::vector<int32_t> &pat = ST.pat;
        SqfLaunch &L = ST.L;
        SqfJob *d_jobs = ST.d_jobs;
        const int stride = ST.stride;
        cudaError_t e = cudaSuccess;
        // ---- lucky primes: largest square-free degree, then the most common pattern
        gbr_parallel_for(nj, threads, [&](int lo, int hi) {
            std::vector<std::pair<uint64_t, int>> cand_slots;
            for (int q = lo; q < hi; ++q) {
                const int j = pend[q];
                SqfJob &x = J[q];
                const int32_t *pq = pat.data() + x.pat_off;
                // slots of the largest square-free degree, grouped by their degree pattern
                int best = -1;
                for (int sl = 0; sl < K; ++sl) {
                    const int32_t *ps = pq + (int64_t)sl * (x.n + 2);
                    if (ps[0] < 1) continue;
                    int sd = 0;
                    for (int i = 0; i < ps[0]; ++i) sd += ps[1 + i];
                    best = std::max(best, sd);
                }
                cand_slots.clear();
                for (int sl = 0; sl < K && best >= 0; ++sl) {
                    const int32_t *ps = pq + (int64_t)sl * (x.n + 2);
                    if (ps[0] < 1) continue;
                    int sd = 0;
                    uint64_t hsh = 1469598103934665603ull;
                    for (int i = 0; i <= ps[0]; ++i) {
                        if (i) sd += ps[i];
                        hsh = (hsh ^ (uint32_t)ps[i]) * 1099511628211ull;
                    }
                    if (sd == best) cand_slots.push_back({hsh, sl});
                }
                std::sort(cand_slots.begin(), cand_slots.end());
                // the longest run of one hash; slots whose pattern differs from the
                // run's first (a hash collision) are left out
                size_t rb = 0, rl = 0;
                for (size_t i = 0; i < cand_slots.size();) {
                    size_t k2 = i;
                    while (k2 < cand_slots.size() && cand_slots[k2].first == cand_slots[i].first) ++k2;
                    if (k2 - i > rl) {
                        rb = i;
                        rl = k2 - i;
                    }
                    i = k2;
                }
                const int32_t *rep = rl ? pq + (int64_t)cand_slots[rb].second * (x.n + 2) : nullptr;
                std::vector<int> &lucky = H[j].lucky;
                lucky.clear();
                for (size_t i = rb; i < rb + rl; ++i) {
                    const int32_t *ps = pq + (int64_t)cand_slots[i].second * (x.n + 2);
                    if (std::equal(ps, ps + 1 + ps[0], rep)) lucky.push_back(cand_slots[i].second);
                }
                std::sort(lucky.begin(), lucky.end());
                const std::vector<int> gpat = rep ? std::vector<int>(rep + 1, rep + 1 + rep[0]) : std::vector<int>();
                const std::vector<int> *gp = rep ? &gpat : nullptr;
                int dmax = 0, nfac = 0;
                if (gp)
                    for (int d : *gp) {
                        dmax = std::max(dmax, d);
                        nfac += d + 1;
                    }
                const int kneed = primes_for_bits(dmax + H[j].l2norm2 + 3.0);
                if (!gp || (int)lucky.size() < kneed) {
                    x.status = 2;
                    continue;
                }
                H[j].pat = *gp;
                lucky.resize(kneed);
                x.status = 0;
                x.lift_k = kneed;
                x.lift_L = (31 * kneed + 31) / 32 + 1;
                x.nfac = nfac;
            }
        });
        std::vector<int> retry, lifted;
        int64_t lsel_w = 0, gtab_w = 0, lift_w = 0, lsign_w = 0, lift_items = 0;
        int KMx = 1, LMx = 1;
        for (int q = 0; q < nj; ++q) {
            SqfJob &x = J[q];
            x.lift0 = lift_items;   // jobs that are not lifted keep an empty range here
            if (x.status != 0) {
                retry.push_back(pend[q]);
                continue;
            }
            lifted.push_back(q);
            x.lsel_off = lsel_w;
            x.gtab_off = gtab_w;
            x.lift_off = lift_w;
            x.lsign_off = lsign_w;
            lsel_w += x.lift_k;
            gtab_w += x.lift_k + (int64_t)x.lift_k * (x.lift_k - 1) / 2;
            lift_w += (int64_t)x.nfac * x.lift_L;
            lsign_w += x.nfac;
            lift_items += x.nfac;
            KMx = std::max(KMx, x.lift_k);
            LMx = std::max(LMx, x.lift_L);
        }
        if (!lifted.empty()) {
            std::vector<int32_t> lsel(lsel_w);
            for (int q : lifted)
                std::memcpy(lsel.data() + J[q].lsel_off, H[pend[q]].lucky.data(), (size_t)J[q].lift_k * 4);
            int32_t *d_lsel = (int32_t *)B.get((size_t)lsel_w * 4);
            uint32_t *d_gtab = (uint32_t *)B.get((size_t)gtab_w * 4);
            uint32_t *d_lift = (uint32_t *)B.get((size_t)lift_w * 4);
            int8_t *d_lsign = (int8_t *)B.get((size_t)lsign_w);
            if (!d_lsel || !d_gtab || !d_lift || !d_lsign)
                return c->fail(GBR_ENOMEM, "device budget too small for the square-free lift");
            L.lsel = d_lsel;
            L.gtab = d_gtab;
            L.lift = d_lift;
            L.lsign = d_lsign;
            e = sqf_copy(c, d_jobs, J.data(), sizeof(SqfJob) * nj, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = sqf_copy(c, d_lsel, lsel.data(), (size_t)lsel_w * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) {
                k_sqf_garner<<<std::min(nj, 1024), 128, 0, s>>>(L);
                e = cudaGetLastError();
                ++c->gcd_kernels;
            }
            int block = 128;
            while (block > 32 && (size_t)(KMx + LMx) * block * 4 > 160 * 1024) block >>= 1;
            const size_t lsm = (size_t)(KMx + LMx) * block * 4;
            if (lsm > kMaxDynSmem) return c->fail(GBR_ELIMIT, "square-free lift needs too many primes");
            if (e == cudaSuccess) {
                k_sqf_lift<<<sqf_blocks((const void *)k_sqf_lift, block, lsm, (lift_items + block - 1) / block), block,
                             lsm, s>>>(L, KMx, LMx, lift_items);
                e = cudaGetLastError();
                ++c->gcd_kernels;
            }
            std::vector<uint32_t> hlift(lift_w);
            std::vector<int8_t> hlsign(lsign_w);
            int32_t herr = 0;
            if (e == cudaSuccess) e = sqf_copy(c, hlift.data(), d_lift, (size_t)lift_w * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = sqf_copy(c, hlsign.data(), d_lsign, (size_t)lsign_w, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = sqf_copy(c, &herr, c->d_err, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "square-free lift", e);
            if (herr) return c->fail(GBR_EDEVICE, "square-free device-side consistency check failed");
            // ---- primitive parts, unit, the check's coefficient bound (per job, in parallel)
            const int nl = (int)lifted.size();
            std::vector<char> okv(nl, 0);
            std::vector<double> bitsv(nl, 0.0);
            gbr_parallel_for(nl, threads, [&](int lo, int hi) {
                bn::Scratch S;
                for (int t = lo; t < hi; ++t) {
                    const int q = lifted[t];
                    SqfHost &h = H[pend[q]];
                    h.fac.assign(h.pat.size(), FlatPoly());
                    bool ok = true;
                    int off = 0;
                    bn::Big lcprod = bn::from_u64(1);
                    for (size_t i = 0; i < h.pat.size() && ok; ++i) {
                        const int d = h.pat[i];
                        ok = primitive_part(hlift.data() + J[q].lift_off + (int64_t)off * J[q].lift_L,
                                            hlsign.data() + J[q].lsign_off + off, d, J[q].lift_L, h.fac[i], S);
                        off += d + 1;
                        if (!ok) break;
                        const bn::Big l = lead(h.fac[i]);
                        for (size_t e3 = 0; e3 <= i; ++e3) lcprod = bn::mul(lcprod, l);
                    }
                    if (ok) ok = bn::divexact(h.lc, lcprod, h.u, S);
                    okv[t] = ok;
                    if (!ok) continue;
                    // coefficient bound of u prod r_i^i: |u| prod ||r_i||_1^i
                    double bits = bn::log2_mag(h.u.m);
                    for (size_t i = 0; i < h.fac.size(); ++i) {
                        const FlatPoly &f = h.fac[i];
                        bits += (double)(i + 1) * log2_norms(f.deg + 1, [&](int k, const uint32_t *&x, size_t &n2) {
                                    x = f.mag.data() + (size_t)k * f.L;
                                    n2 = f.sign[k] ? bn::top(x, (size_t)f.L) : 0;
                                }).l1;
                    }
                    bitsv[t] = std::max(bits, h.l2inf) + 2.0;
                }
            });
            std::vector<int> cand;
            double maxbits_v = 0.0;
            for (int t = 0; t < nl; ++t) {
                if (!okv[t]) {
                    retry.push_back(pend[lifted[t]]);
                    continue;
                }
                cand.push_back(lifted[t]);
                maxbits_v = std::max(maxbits_v, bitsv[t]);
            }
            // ---- exact check: R = u prod r_i^i modulo enough primes
            if (!cand.empty()) {
                const int Kv = primes_for_bits(maxbits_v);
                if (Kv > NP) return c->fail(GBR_ELIMIT, "square-free check needs more than the table's primes");
                const int nv = (int)cand.size();
                int VL = 1, maxfac = 1;
                std::vector<int64_t> voff(nv + 1, 0);
                for (int t = 0; t < nv; ++t) {
                    const SqfHost &h = H[pend[cand[t]]];
                    VL = std::max(VL, (int)h.u.m.size());
                    for (const auto &f : h.fac) VL = std::max(VL, f.L);
                    maxfac = std::max(maxfac, (int)h.fac.size());
                }
                std::vector<SqfJob> JV(nv);
                int64_t vres = 0;
                for (int t = 0; t < nv; ++t) {
                    const SqfHost &h = H[pend[cand[t]]];
                    int ncoef = 1;
                    for (const auto &f : h.fac) ncoef += f.deg + 1;
                    SqfJob x = J[cand[t]];
                    x.status = 0;
                    x.res_off = vres;
                    x.red0 = vres;
                    x.ver_L = VL;
                    x.nfac = (int)h.fac.size();
                    x.ver_off = voff[t];
                    vres += (int64_t)Kv * (x.n + 1);
                    voff[t + 1] = voff[t] + (int64_t)ncoef * VL + (ncoef + 3) / 4;
                    JV[t] = x;
                }
                std::vector<uint32_t> hv(voff[nv], 0u);
                std::vector<int32_t> hdeg((size_t)nv * (maxfac + 1), 0);
                gbr_parallel_for(nv, threads, [&](int lo, int hi) {
                    for (int t = lo; t < hi; ++t) {
                        const SqfHost &h = H[pend[cand[t]]];
                        uint32_t *w = hv.data() + voff[t];
                        int ncoef = 1;
                        for (const auto &f : h.fac) ncoef += f.deg + 1;
                        int8_t *sg = reinterpret_cast<int8_t *>(w + (int64_t)ncoef * VL);
                        std::copy(h.u.m.begin(), h.u.m.end(), w);
                        sg[0] = (int8_t)h.u.s;
                        int k = 1;
                        for (size_t i = 0; i < h.fac.size(); ++i) {
                            const FlatPoly &f = h.fac[i];
                            hdeg[(size_t)t * (maxfac + 1) + i] = f.deg;
                            for (int e2 = 0; e2 <= f.deg; ++e2, ++k) {
                                std::copy(f.mag.begin() + (size_t)e2 * f.L, f.mag.begin() + (size_t)(e2 + 1) * f.L,
                                          w + (int64_t)k * VL);
                                sg[k] = f.sign[e2];
                            }
                        }
                    }
                });
                SqfJob *d_jv = (SqfJob *)B.get(sizeof(SqfJob) * nv);
                uint32_t *d_vres = (uint32_t *)B.get((size_t)vres * 4);
                uint32_t *d_ver = (uint32_t *)B.get(hv.size() * 4);
                int32_t *d_vdeg = (int32_t *)B.get(hdeg.size() * 4);
                int32_t *d_fail = (int32_t *)B.get((size_t)nv * 4);
                if (!d_jv || !d_vres || !d_ver || !d_vdeg || !d_fail)
                    return c->fail(GBR_ENOMEM, "device budget too small for the square-free check");
                SqfLaunch V = L;
                V.jobs = d_jv;
                V.njobs = nv;
                V.p0 = 0;
                V.nprimes = Kv;
                V.res = d_vres;
                V.ver = d_ver;
                V.ver_deg = d_vdeg;
                V.ver_fail = d_fail;
                V.max_fac = maxfac;
                e = sqf_copy(c, d_jv, JV.data(), sizeof(SqfJob) * nv, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = sqf_copy(c, d_ver, hv.data(), hv.size() * 4, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = sqf_copy(c, d_vdeg, hdeg.data(), hdeg.size() * 4, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaMemsetAsync(d_fail, 0, (size_t)nv * 4, s);
                if (e == cudaSuccess) {
                    k_sqf_reduce<<<sqf_blocks((const void *)k_sqf_reduce, 256, 0, (vres + 255) / 256), 256, 0, s>>>(V, vres);
                    e = cudaGetLastError();
                    ++c->gcd_kernels;
                }
                const int nwv = sqf_warps(3, stride);
                if (nwv < 1) return c->fail(GBR_ELIMIT, "square-free input degree too large for shared memory");
                if (e == cudaSuccess) {
                    const size_t smem = (size_t)nwv * 3 * stride * 4;
                    k_sqf_verify<<<sqf_blocks((const void *)k_sqf_verify, nwv * 32, smem,
                                              ((int64_t)nv * Kv + nwv - 1) / nwv),
                                   nwv * 32, smem, s>>>(V, stride);
                    e = cudaGetLastError();
                    ++c->gcd_kernels;
                    c->gcd_subproblems += (int64_t)nv * Kv;
                }
                std::vector<int32_t> fail(nv);
                if (e == cudaSuccess) e = sqf_copy(c, fail.data(), d_fail, (size_t)nv * 4, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "square-free check", e);
                for (int t = 0; t < nv; ++t) {
                    const int j = pend[cand[t]];
                    if (fail[t]) retry.push_back(j);
                    else H[j].status = 1;
                }
            }
        }
        pend = retry;
        std::sort(pend.begin(), pend.end());
        pend.erase(std::unique(pend.begin(), pend.end()), pend.end());
        K *= 2;
    }
    // ---- results: the units and factors of all inputs share one refcounted host block
    std::vector<int64_t> roff(n + 1, 0);
    for (int j = 0; j < n; ++j) roff[j + 1] = roff[j] + 1 + (int64_t)H[j].fac.size();
    std::vector<gbr_bigpoly> res(roff[n]);
    for (int j = 0; j < n; ++j) {
        const SqfHost &h = H[j];
        gbr_bigpoly *r = res.data() + roff[j];
        r[0].deg = h.u.s ? 0 : -1;
        r[0].limbs = std::max<int>(1, (int)h.u.m.size());
        for (size_t i = 0; i < h.fac.size(); ++i) {
            r[1 + i].deg = h.fac[i].deg;
            r[1 + i].limbs = h.fac[i].L;
        }
    }
    for (int j = 0; j < n; ++j)
        if (!H[j].fac.empty()) {
            out[j].factors = (gbr_bigpoly *)std::malloc(sizeof(gbr_bigpoly) * H[j].fac.size());
            if (!out[j].factors) return c->fail(GBR_ENOMEM, "host result allocation");
            out[j].count = (int32_t)H[j].fac.size();
            for (int i = 0; i < out[j].count; ++i) out[j].factors[i] = gbr_bigpoly{-1, 0, nullptr, nullptr};
        }
    if (!gbr_alloc_results(res.data(), (int)res.size())) return c->fail(GBR_ENOMEM, "host result allocation");
    gbr_parallel_for(n, threads, [&](int lo, int hi) {
        for (int j = lo; j < hi; ++j) {
            const SqfHost &h = H[j];
            gbr_bigpoly *r = res.data() + roff[j];
            if (h.u.s) {
                for (int l = 0; l < r[0].limbs; ++l) r[0].mag[l] = l < (int)h.u.m.size() ? h.u.m[l] : 0u;
                r[0].sign[0] = (int8_t)h.u.s;
            }
            for (size_t i = 0; i < h.fac.size(); ++i) {
                std::copy(h.fac[i].mag.begin(), h.fac[i].mag.end(), r[1 + i].mag);
                std::copy(h.fac[i].sign.begin(), h.fac[i].sign.end(), r[1 + i].sign);
                out[j].factors[i] = r[1 + i];
            }
            out[j].unit = r[0];
        }
    });
    return GBR_OK;
}

extern "C" int gbr_squarefree_batch(gbr_ctx *c, int n, const gbr_bigpoly *in, gbr_sqf *out) {
    if (!c || n < 0 || (n && (!in || !out))) return GBR_EINVAL;
    for (int j = 0; j < n; ++j) {
        out[j].unit.deg = -1;
        out[j].unit.limbs = 0;
        out[j].unit.mag = nullptr;
        out[j].unit.sign = nullptr;
        out[j].count = 0;
        out[j].factors = nullptr;
    }
    if (n == 0) return GBR_OK;
    NvtxScope call("gbr_squarefree_batch");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    int st;
    const auto t0 = std::chrono::steady_clock::now();
    if (c->stats_on) cudaEventRecord(c->ev[0], c->stream);
    try {
        st = sqf_batch_locked(c, n, in, out);
        if (c->stats_on) {
            // the whole call on the context's stream, as for a gcd call
            cudaEventRecord(c->ev[1], c->stream);
            cudaEventSynchronize(c->ev[1]);
            gbr_stats g{};
            float ms = 0;
            cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
            g.gcd_ms = ms;
            g.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            g.kernels = c->gcd_kernels;
            g.subproblems = c->gcd_subproblems;
            g.h2d_bytes = c->gcd_h2d;
            g.d2h_bytes = c->gcd_d2h;
            c->stats = g;
        }
    } catch (std::bad_alloc &) {
        st = c->fail(GBR_ENOMEM, "host allocation");
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (st)
        for (int j = 0; j < n; ++j) gbr_free_sqf(c, &out[j]);
    return st;
}

extern "C" int gbr_squarefree(gbr_ctx *c, const gbr_bigpoly *in, gbr_sqf *out) {
    if (!in || !out) return GBR_EINVAL;
    return gbr_squarefree_batch(c, 1, in, out);
}

extern "C" void gbr_free_sqf(gbr_ctx *c, gbr_sqf *x) {
    if (!x) return;
    gbr_free_result(c, &x->unit);
    if (x->factors) {
        for (int i = 0; i < x->count; ++i) gbr_free_result(c, &x->factors[i]);
        std::free(x->factors);
    }
    x->factors = nullptr;
    x->count = 0;
}

cudaError_t gbr::configure_sqf_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_sqf_yun, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sqf_lift, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sqf_verify, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    return e;
}
