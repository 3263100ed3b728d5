// Exact gcd of univariate integer polynomials, multi-modular.
//
// Section 4 ("Symbolic Speedups") of the paper runs univariate gcds on the GPU
// with the same divide-conquer-combine scheme as the resultant (modular images,
// solve over F_p, Chinese remaindering) and notes that one moderate-degree gcd
// has too little parallelism; batching many gcds supplies it.
//
// Method (small-primes modular gcd with an exact certificate):
//   prep     one warp per job: degrees, contents cP, cQ, c = gcd(cP, cQ),
//            b = gcd(lc(P/cP), lc(Q/cQ)), log2 of the bound B below
//   modp     one warp per (job, prime): P' = P/cP and Q' = Q/cQ mod p, Euclid
//            (fraction-free steps), G_p = monic gcd, then w = b G_p and the exact
//            cofactors f = P'/G_p, g = Q'/G_p
//   (host)   keep the primes whose gcd degree is minimal
//   crt      Garner lift of w, f, g with symmetric residues
//   check    ||f||_1 ||w||_1 < M/2 and ||g||_1 ||w||_1 < M/2 prove f w = b P' and
//            g w = b Q' over Z (both sides agree mod M and are below M/2), so
//            pp(w) divides P' and Q'; its degree is the minimal modular degree,
//            which no common divisor exceeds, so pp(w) = gcd(P', Q').  Result:
//            c * pp(w), with cont(w) = gcd(b, coefficients of w) since lc(w) = b.
//   The prime count makes M > 2 b max(2^dP ||P'||_2, 2^dQ ||Q'||_2), which bounds
//   ||f||_1 ||w||_1 for the true factors (Landau: Mahler measure <= 2-norm), so the
//   check can only fail when every chosen prime was unlucky; then more primes
//   are taken.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include <chrono>

#include "gbr_core.h"

namespace gbr {

struct GcdInfo {
    int32_t dP, dQ;
    int64_t lcP, lcQ;
    uint64_t cP, cQ, c, b;
    double log2B;
};

struct GcdPlan {
    int32_t dP, dQ, nslots, kcrt;
    int32_t S, Lcrt, Lout, status;      // status: 0 pending, 1 ok, 2 check failed
    int64_t pin_off, qin_off;           // int64 words of P and Q in the input buffer
    int64_t slot_off;                   // residues: slot s at slot_off + s*S
    int64_t slotlist_off;               // int32 prime-table index per slot
    int64_t crtlist_off;                // int32 slot index per CRT prime
    int64_t garner_off;                 // kcrt + kcrt(kcrt-1)/2 words
    int64_t lift_off, lsign_off;        // lifted w|f|g limbs and signs
    int64_t out_off, osign_off;         // final result limbs and signs
    int64_t cof_off, cofsign_off;       // cofactors P/G then Q/G (Lcof limbs each), when asked for
    int32_t dstar, Lcof;
    uint64_t cP, cQ, c, b;
    double log2M;
};

struct GcdLaunch {
    const int64_t *in;
    const int64_t *in_off;   // per job: offset of P; Q follows at in_off + dPext + 1
    const int32_t *in_deg;   // per job: extents (deg P, deg Q) pairs
    GcdInfo *info;
    const GcdPlan *plan;
    const ModP *mods;
    uint32_t *slots;
    int32_t *slotlist;       // also carries, at the same index in `sdeg`, the slot's gcd degree
    int32_t *sdeg;
    const int32_t *crtlist;
    uint32_t *garner;
    uint32_t *lift;
    int8_t *lsign;
    uint32_t *out;
    int8_t *osign;
    int32_t *odeg;
    uint32_t *cof;           // optional cofactor outputs (null: gcd only)
    int8_t *cofsign;
    int32_t *status;
    int32_t *err;
    int32_t njobs;
};

__device__ __forceinline__ uint64_t gcd_u64(uint64_t a, uint64_t b) {
    if (!a) return b;
    if (!b) return a;
    int s = __ffsll((long long)(a | b)) - 1;
    a >>= __ffsll((long long)a) - 1;
    while (b) {
        b >>= __ffsll((long long)b) - 1;
        if (a > b) {
            uint64_t t = a;
            a = b;
            b = t;
        }
        b -= a;
    }
    return a << s;
}

__device__ __forceinline__ uint64_t uabs64(int64_t v) { return v < 0 ? 0ull - (uint64_t)v : (uint64_t)v; }

__device__ __forceinline__ uint32_t mp_from_u64(uint64_t u, const ModP &M) {
    uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    return mp_add(mp_mul(mp_to(hi, M), M.r2, M), mp_to(lo, M), M.p);
}

__device__ __forceinline__ uint32_t mp_from_i64(int64_t v, const ModP &M) {
    uint32_t r = mp_from_u64(uabs64(v), M);
    return v < 0 ? mp_neg(r, M.p) : r;
}

__device__ __forceinline__ int wl_find_g(const int64_t *start, int n, int64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ prep

__global__ void k_gcd_prep(GcdLaunch L) {
    int job = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (job >= L.njobs) return;
    const int64_t *P = L.in + L.in_off[job];
    int eP = L.in_deg[2 * job], eQ = L.in_deg[2 * job + 1];
    const int64_t *Q = P + eP + 1;
    GcdInfo I;
    int d[2];
    uint64_t cont[2];
    double l2[2];   // log2 ||.||_2
    for (int w = 0; w < 2; ++w) {
        const int64_t *X = w ? Q : P;
        int e = w ? eQ : eP;
        int dd = -1;
        uint64_t g = 0;
        double mx = -INFINITY, s = 0.0;
        for (int i = lane; i <= e; i += 32) {
            int64_t v = X[i];
            if (v) {
                dd = i;
                uint64_t a = uabs64(v);
                g = gcd_u64(g, a);
                double lv = 2.0 * log2((double)a);
                if (lv > mx) { s = s * exp2(mx - lv) + 1.0; mx = lv; }
                else s += exp2(lv - mx);
            }
        }
        for (int o = 16; o; o >>= 1) {
            dd = max(dd, __shfl_xor_sync(0xffffffffu, dd, o));
            g = gcd_u64(g, __shfl_xor_sync(0xffffffffu, g, o));
            double omx = __shfl_xor_sync(0xffffffffu, mx, o), os = __shfl_xor_sync(0xffffffffu, s, o);
            if (os != 0.0) {
                if (s == 0.0) { mx = omx; s = os; }
                else if (omx > mx) { s = s * exp2(mx - omx) + os; mx = omx; }
                else s += os * exp2(omx - mx);
            }
        }
        d[w] = dd;
        cont[w] = g;
        l2[w] = s == 0.0 ? -INFINITY : 0.5 * (mx + log2(s));
    }
    I.dP = d[0];
    I.dQ = d[1];
    I.lcP = d[0] >= 0 ? P[d[0]] : 0;
    I.lcQ = d[1] >= 0 ? Q[d[1]] : 0;
    I.cP = cont[0];
    I.cQ = cont[1];
    I.c = gcd_u64(cont[0], cont[1]);
    uint64_t lp = d[0] >= 0 ? uabs64(I.lcP) / cont[0] : 0, lq = d[1] >= 0 ? uabs64(I.lcQ) / cont[1] : 0;
    I.b = gcd_u64(lp, lq);
    double bp = d[0] >= 0 ? d[0] + l2[0] - log2((double)cont[0]) : -INFINITY;
    double bq = d[1] >= 0 ? d[1] + l2[1] - log2((double)cont[1]) : -INFINITY;
    I.log2B = (I.b ? log2((double)I.b) : 0.0) + fmax(bp, bq);
    if (lane == 0) L.info[job] = I;
}

// ------------------------------------------------------------------ per-prime gcd and cofactors

__global__ void k_gcd_modp(GcdLaunch L, const int64_t *wl_start, const int32_t *wl_jobs, int wl_n, int64_t total,
                           int regw) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t *R0 = smem + (size_t)wid * 2 * regw;
    uint32_t *R1 = R0 + regw;
    for (int64_t item = (int64_t)blockIdx.x * nw + wid; item < total; item += (int64_t)gridDim.x * nw) {
        int bi = wl_find_g(wl_start, wl_n, item);
        int job = wl_jobs[bi];
        int slot = (int)(item - wl_start[bi]);
        const GcdPlan &G = L.plan[job];
        const int64_t *P = L.in + G.pin_off;
        const int64_t *Q = L.in + G.qin_off;
        const ModP M = L.mods[L.slotlist[G.slotlist_off + slot]];
        const uint32_t icp = mp_inv(mp_from_u64(G.cP, M), M), icq = mp_inv(mp_from_u64(G.cQ, M), M);
        for (int t = lane; t <= G.dP; t += 32) R0[t] = mp_mul(mp_from_i64(P[t], M), icp, M);
        for (int t = lane; t <= G.dQ; t += 32) R1[t] = mp_mul(mp_from_i64(Q[t], M), icq, M);
        __syncwarp();
        uint32_t *A = R0, *B = R1;
        int da = G.dP, db = G.dQ;
        while (da >= 0 && A[da] == 0) --da;
        while (db >= 0 && B[db] == 0) --db;
        // Euclid with fraction-free steps A <- lc(B) A - lc(A) x^(da-db) B
        while (db >= 0) {
            if (da < db) {
                uint32_t *t = A; A = B; B = t;
                int ti = da; da = db; db = ti;
                continue;
            }
            const uint32_t zeta = B[db], q = A[da];
            const int s = da - db;
            for (int t = lane; t < da; t += 32)
                A[t] = t >= s ? mp_mulsub(zeta, A[t], q, B[t - s], M) : mp_mul(zeta, A[t], M);
            __syncwarp();
            --da;
            while (da >= 0 && A[da] == 0) --da;
        }
        // A holds the gcd (degree da >= 0: P', Q' are non-zero mod p); make it monic
        const int d = da;
        const uint32_t il = mp_inv(A[d], M);
        __syncwarp();
        for (int t = lane; t <= d; t += 32) A[t] = mp_mul(A[t], il, M);
        __syncwarp();
        uint32_t *T = B;   // B is zero now; reuse its region for the divisions
        uint32_t *out = L.slots + G.slot_off + (int64_t)slot * G.S;
        const int mn = min(G.dP, G.dQ);
        const uint32_t bt = mp_from_u64(G.b, M);
        for (int t = lane; t <= d; t += 32) out[t] = mp_from(mp_mul(A[t], bt, M), M);
        for (int w = 0; w < 2; ++w) {
            const int64_t *X = w ? Q : P;
            const int dx = w ? G.dQ : G.dP;
            const uint32_t ic = w ? icq : icp;
            for (int t = lane; t <= dx; t += 32) T[t] = mp_mul(mp_from_i64(X[t], M), ic, M);
            __syncwarp();
            for (int k = dx; k >= d; --k) {
                const uint32_t qk = T[k];
                for (int t = lane; t < d; t += 32) T[k - d + t] = mp_sub(T[k - d + t], mp_mul(qk, A[t], M), M.p);
                __syncwarp();
            }
            for (int t = lane; t < d; t += 32)
                if (T[t] != 0u) atomicExch(L.err, 3);
            uint32_t *o = out + (mn + 1) + (w ? G.dP + 1 : 0);
            for (int t = lane; t <= dx - d; t += 32) o[t] = mp_from(T[d + t], M);
            __syncwarp();
        }
        if (lane == 0) L.sdeg[G.slotlist_off + slot] = d;
    }
}

// ------------------------------------------------------------------ Garner tables per job list

__global__ void k_gcd_garner(GcdLaunch L, const int32_t *jobs, int njobs) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    // thread t handles (job index t / 2048? ) -- one thread per (job, i) pair via grid-stride
    for (int64_t it = t; it < (int64_t)njobs * GBR_MAX_PRIMES; it += (int64_t)gridDim.x * blockDim.x) {
        int ji = (int)(it / GBR_MAX_PRIMES), i = (int)(it % GBR_MAX_PRIMES);
        const GcdPlan &G = L.plan[jobs[ji]];
        if (i >= G.kcrt) continue;
        const int32_t *cl = L.crtlist + G.crtlist_off;
        const int32_t *sl = L.slotlist + G.slotlist_off;
        const ModP M = L.mods[sl[cl[i]]];
        uint32_t *tab = L.garner + G.garner_off;
        uint32_t *pm = tab + G.kcrt + (int64_t)i * (i - 1) / 2;
        uint32_t prod = M.r1;
        for (int j = 0; j < i; ++j) {
            uint32_t pj = L.mods[sl[cl[j]]].p;
            pj = min(pj, pj - M.p);
            uint32_t pjm = mp_to(pj, M);
            pm[j] = pjm;
            prod = mp_mul(prod, pjm, M);
        }
        tab[i] = mp_inv(prod, M);
    }
}

// ------------------------------------------------------------------ Garner lift of w | f | g

__global__ void k_gcd_crt(GcdLaunch L, const int64_t *wl_start, const int32_t *wl_jobs, int wl_n, int64_t total,
                          int LM) {
    extern __shared__ uint32_t smem[];
    const int BS = blockDim.x;
    uint32_t *limb = smem + threadIdx.x;
    for (int64_t item = blockIdx.x * (int64_t)BS + threadIdx.x; item < total; item += (int64_t)gridDim.x * BS) {
        int bi = wl_find_g(wl_start, wl_n, item);
        int job = wl_jobs[bi];
        int e = (int)(item - wl_start[bi]);
        const GcdPlan &G = L.plan[job];
        const int d = G.dstar, mn = min(G.dP, G.dQ);
        int pos;
        if (e <= d) pos = e;
        else if (e <= d + (G.dP - d + 1)) pos = (mn + 1) + (e - d - 1);
        else pos = (mn + 1) + (G.dP + 1) + (e - d - 1 - (G.dP - d + 1));
        const int32_t *cl = L.crtlist + G.crtlist_off;
        const int32_t *sl = L.slotlist + G.slotlist_off;
        const uint32_t *tab = L.garner + G.garner_off;
        const int k = G.kcrt;
        uint32_t *base = L.slots + G.slot_off + pos;
        auto V = [&](int i) -> uint32_t & { return base[(int64_t)cl[i] * G.S]; };
        for (int i = 1; i < k; ++i) {
            const ModP M = L.mods[sl[cl[i]]];
            const uint32_t *pmi = tab + k + (int64_t)i * (i - 1) / 2;
            uint32_t t = V(i - 1);
            t = min(t, t - M.p);
            for (int j = i - 2; j >= 0; --j) {
                uint32_t vj = V(j);
                vj = min(vj, vj - M.p);
                t = mp_add(mp_mul(t, pmi[j], M), vj, M.p);
            }
            V(i) = mp_mul(mp_sub(V(i), t, M.p), tab[i], M);
        }
        int cmp = 0;
        for (int i = k - 1; i >= 0 && cmp == 0; --i) {
            uint32_t dg = V(i), h = (L.mods[sl[cl[i]]].p - 1u) >> 1;
            cmp = (dg > h) - (dg < h);
        }
        const bool neg = cmp > 0;
        int nl = 0;
        for (int i = k - 1; i >= 0; --i) {
            const uint32_t p = L.mods[sl[cl[i]]].p;
            uint32_t dg = V(i);
            if (neg) dg = p - 1u - dg;
            uint32_t carry = dg;
            for (int l = 0; l < nl; ++l) {
                uint64_t t = (uint64_t)limb[l * BS] * p + carry;
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
        uint32_t *o = L.lift + G.lift_off + (int64_t)e * G.Lcrt;
        for (int l = 0; l < G.Lcrt; ++l) o[l] = l < nl ? limb[l * BS] : 0u;
        L.lsign[G.lsign_off + e] = nl == 0 ? 0 : (neg ? -1 : 1);
    }
}

// ------------------------------------------------------------------ certificate and normalisation

__device__ double limbs_log2(const uint32_t *x, int n) {
    int t = n - 1;
    while (t >= 0 && x[t] == 0) --t;
    if (t < 0) return -INFINITY;
    double v = (double)x[t];
    if (t >= 1) v += (double)x[t - 1] * 0x1p-32;
    if (t >= 2) v += (double)x[t - 2] * 0x1p-64 + 0x1p-64;   // round the truncated tail up
    return log2(v) + 32.0 * t + 1e-12;
}

__device__ uint64_t limbs_mod(const uint32_t *x, int n, uint64_t m) {
    unsigned __int128 r = 0;
    for (int l = n - 1; l >= 0; --l) r = ((r << 32) | x[l]) % m;
    return (uint64_t)r;
}

__global__ void k_gcd_check(GcdLaunch L, const int32_t *jobs, int njobs) {
    int wj = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (wj >= njobs) return;
    const int job = jobs[wj];
    const GcdPlan &G = L.plan[job];
    const int d = G.dstar;
    const int nw = d + 1, nf = G.dP - d + 1, ng = G.dQ - d + 1;
    const uint32_t *lift = L.lift + G.lift_off;
    double nrm[3];
    for (int part = 0; part < 3; ++part) {
        int first = part == 0 ? 0 : (part == 1 ? nw : nw + nf);
        int cnt = part == 0 ? nw : (part == 1 ? nf : ng);
        double mx = -INFINITY, s = 0.0;
        for (int i = lane; i < cnt; i += 32) {
            double a = limbs_log2(lift + (int64_t)(first + i) * G.Lcrt, G.Lcrt);
            if (a == -INFINITY) continue;
            if (a > mx) { s = s * exp2(mx - a) + 1.0; mx = a; }
            else s += exp2(a - mx);
        }
        for (int o = 16; o; o >>= 1) {
            double omx = __shfl_xor_sync(0xffffffffu, mx, o), os = __shfl_xor_sync(0xffffffffu, s, o);
            if (os != 0.0) {
                if (s == 0.0) { mx = omx; s = os; }
                else if (omx > mx) { s = s * exp2(mx - omx) + os; mx = omx; }
                else s += os * exp2(omx - mx);
            }
        }
        nrm[part] = s == 0.0 ? -INFINITY : mx + log2(s) * (1.0 + 1e-12) + 1e-9;
    }
    const double lim = G.log2M - 1.0 - 1e-6;
    bool ok = nrm[0] + nrm[1] < lim && nrm[0] + nrm[2] < lim;
    // the leading coefficient of w must be exactly b (positive)
    if (ok) {
        const uint32_t *lw = lift + (int64_t)d * G.Lcrt;
        ok = L.lsign[G.lsign_off + d] > 0 && (uint32_t)G.b == lw[0] && (uint32_t)(G.b >> 32) == (G.Lcrt > 1 ? lw[1] : 0u);
        for (int l = 2; l < G.Lcrt; ++l) ok = ok && lw[l] == 0u;
    }
    if (!ok) {
        if (lane == 0) L.status[job] = 2;
        return;
    }
    // content of w divides b: gcd(b, |w_i| mod b) over all coefficients
    uint64_t g = G.b;
    for (int i = lane; i < nw; i += 32) g = gcd_u64(g, limbs_mod(lift + (int64_t)i * G.Lcrt, G.Lcrt, G.b));
    for (int o = 16; o; o >>= 1) g = gcd_u64(g, __shfl_xor_sync(0xffffffffu, g, o));
    // result coefficient i = c * |w_i| / g with the sign of w_i
    for (int i = lane; i < nw; i += 32) {
        const uint32_t *x = lift + (int64_t)i * G.Lcrt;
        uint32_t *o = L.out + G.out_off + (int64_t)i * G.Lout;
        unsigned __int128 r = 0;
        for (int l = G.Lcrt - 1; l >= 0; --l) {
            r = (r << 32) | x[l];
            o[l] = (uint32_t)(r / g);
            r %= g;
        }
        for (int l = G.Lcrt; l < G.Lout; ++l) o[l] = 0u;
        unsigned __int128 carry = 0;
        for (int l = 0; l < G.Lout; ++l) {
            unsigned __int128 t = (unsigned __int128)o[l] * G.c + carry;
            o[l] = (uint32_t)t;
            carry = t >> 32;
        }
        if (carry) atomicExch(L.err, 4);
        L.osign[G.osign_off + i] = L.lsign[G.lsign_off + i];
    }
    // cofactors P / G = (cP / c) f* / (b / g) and Q / G = (cQ / c) g* / (b / g): from
    // f* w = b P' with w = g pp(w) and G = c pp(w); the divisions are exact
    if (L.cof) {
        const uint64_t lpw = G.b / g;
        for (int part = 0; part < 2; ++part) {
            const int first = part ? nw + nf : nw, cnt = part ? ng : nf, ob = part ? nf : 0;
            const uint64_t cs = (part ? G.cQ : G.cP) / G.c;
            for (int i = lane; i < cnt; i += 32) {
                const uint32_t *x = lift + (int64_t)(first + i) * G.Lcrt;
                uint32_t *o = L.cof + G.cof_off + (int64_t)(ob + i) * G.Lcof;
                unsigned __int128 r = 0;
                for (int l = G.Lcrt - 1; l >= 0; --l) {
                    r = (r << 32) | x[l];
                    o[l] = (uint32_t)(r / lpw);
                    r %= lpw;
                }
                if (r) atomicExch(L.err, 5);
                for (int l = G.Lcrt; l < G.Lcof; ++l) o[l] = 0u;
                unsigned __int128 carry = 0;
                for (int l = 0; l < G.Lcof; ++l) {
                    const unsigned __int128 t = (unsigned __int128)o[l] * cs + carry;
                    o[l] = (uint32_t)t;
                    carry = t >> 32;
                }
                if (carry) atomicExch(L.err, 4);
                L.cofsign[G.cofsign_off + ob + i] = L.lsign[G.lsign_off + first + i];
            }
        }
    }
    if (lane == 0) {
        L.odeg[job] = d;
        L.status[job] = 1;
    }
}

cudaError_t configure_gcd_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_gcd_modp, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gcd_crt, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    return e;
}

}  // namespace gbr

using namespace gbr;

// ------------------------------------------------------------------ host orchestration

namespace {

struct HostGcdJob {
    int dP, dQ;
    GcdInfo info;
    int kneed;
    int status;   // 0 pending, 1 done (device), 2 trivial (host), 3 failed
    int result_src;
};

int grid_for(const void *kernel, int block, size_t smem, int64_t blocks_needed) {
    int per_sm = 0, dev = 0, sms = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t cap = (int64_t)std::max(per_sm, 1) * sms;
    return (int)std::max<int64_t>(1, std::min(cap, blocks_needed));
}

void set_big_int(gbr_bigpoly &b, const std::vector<std::pair<uint64_t, int>> &coef) {
    // coef: (magnitude <= 2^64-1, sign) per power, already trimmed
    b.deg = (int)coef.size() - 1;
    b.limbs = 2;
    b.mag = nullptr;
    b.sign = nullptr;
    if (b.deg < 0) return;
    if (!gbr_alloc_results(&b, 1)) return;
    for (size_t i = 0; i < coef.size(); ++i) {
        b.mag[2 * i] = (uint32_t)coef[i].first;
        b.mag[2 * i + 1] = (uint32_t)(coef[i].first >> 32);
        b.sign[i] = (int8_t)coef[i].second;
    }
}

}  // namespace

// copies of the gcd path, counted for gbr_stats
static cudaError_t gcd_copy(gbr_ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                            cudaStream_t s) {
    if (kind == cudaMemcpyHostToDevice) c->gcd_h2d += (int64_t)bytes;
    else c->gcd_d2h += (int64_t)bytes;
    return cudaMemcpyAsync(dst, src, bytes, kind, s);
}

// out_a, out_b (both or neither): the cofactors p / gcd and q / gcd
static int gcd_batch_locked(gbr_ctx *c, int n, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *out,
                            gbr_bigpoly *out_a = nullptr, gbr_bigpoly *out_b = nullptr) {
    const bool cof = out_a && out_b;
    cudaStream_t s = c->stream;
    cudaError_t e;
    c->gcd_kernels = c->gcd_subproblems = c->gcd_h2d = c->gcd_d2h = 0;
    // ---- validate and pack
    std::vector<int64_t> in_off(n);
    std::vector<int32_t> in_deg(2 * (size_t)n);
    int64_t words = 0;
    for (int i = 0; i < n; ++i) {
        for (const gbr_upoly *u : {&p[i], &q[i]}) {
            if (!u->coef || u->deg < 0) return c->fail(GBR_EINVAL, "bad univariate polynomial");
            if (u->words != 1) return c->fail(GBR_EINVAL, "gcd inputs must have int64 coefficients (words = 1)");
            if (u->deg > GBR_MAX_UDEG) return c->fail(GBR_ELIMIT, "gcd input degree above GBR_MAX_UDEG");
        }
        in_off[i] = words;
        in_deg[2 * i] = p[i].deg;
        in_deg[2 * i + 1] = q[i].deg;
        words += p[i].deg + 1 + q[i].deg + 1;
    }
    int64_t *hin = (int64_t *)c->pinned((size_t)words * 8 + 64, 0);
    if (!hin) return c->fail(GBR_ENOMEM, "pinned host staging");
    for (int i = 0; i < n; ++i) {
        std::memcpy(hin + in_off[i], p[i].coef, (size_t)(p[i].deg + 1) * 8);
        std::memcpy(hin + in_off[i] + p[i].deg + 1, q[i].coef, (size_t)(q[i].deg + 1) * 8);
    }
    struct Bufs {
        gbr_ctx *c;
        std::vector<void *> v;
        void *get(size_t b) {
            void *x = c->dalloc(b ? b : 8);
            if (x) v.push_back(x);
            return x;
        }
        ~Bufs() {
            if (c->stream) cudaStreamSynchronize(c->stream);
            for (void *x : v) c->dfree(x);
        }
    } bufs{c, {}};
    int64_t *d_in = (int64_t *)bufs.get((size_t)words * 8);
    int64_t *d_off = (int64_t *)bufs.get((size_t)n * 8);
    int32_t *d_deg = (int32_t *)bufs.get((size_t)n * 8);
    GcdInfo *d_info = (GcdInfo *)bufs.get(sizeof(GcdInfo) * n);
    if (!d_in || !d_off || !d_deg || !d_info) return c->fail(GBR_ENOMEM, "device budget too small for the gcd batch");
    e = gcd_copy(c, d_in, hin, (size_t)words * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = gcd_copy(c, d_off, in_off.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = gcd_copy(c, d_deg, in_deg.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s);
    GcdLaunch L{};
    L.in = d_in;
    L.in_off = d_off;
    L.in_deg = d_deg;
    L.info = d_info;
    L.mods = c->d_mods;
    L.err = c->d_err;
    L.njobs = n;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, 4, s);
    if (e == cudaSuccess) {
        k_gcd_prep<<<(n * 32 + 127) / 128, 128, 0, s>>>(L);
        c->gcd_kernels++;
        e = cudaGetLastError();
    }
    std::vector<GcdInfo> info(n);
    if (e == cudaSuccess) e = gcd_copy(c, info.data(), d_info, sizeof(GcdInfo) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "gcd prep", e);
    // ---- trivial jobs on the host (zero inputs, constants)
    std::vector<int> pending;
    for (int i = 0; i < n; ++i) {
        const GcdInfo &I = info[i];
        out[i].deg = -1;
        out[i].limbs = 0;
        out[i].mag = nullptr;
        out[i].sign = nullptr;
        if (cof) out_a[i] = out_b[i] = gbr_bigpoly{-1, 0, nullptr, nullptr};
        if (I.dP < 0 && I.dQ < 0) continue;
        if (I.dP < 0 || I.dQ < 0) {   // gcd(X, 0) = X / sign(lc X)
            const int64_t *X = I.dP < 0 ? hin + in_off[i] + p[i].deg + 1 : hin + in_off[i];
            int dx = I.dP < 0 ? I.dQ : I.dP;
            int sg = X[dx] < 0 ? -1 : 1;
            std::vector<std::pair<uint64_t, int>> co(dx + 1);
            for (int t = 0; t <= dx; ++t) {
                int64_t v = X[t];
                uint64_t mag = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
                co[t] = {mag, v == 0 ? 0 : (v < 0 ? -sg : sg)};
            }
            set_big_int(out[i], co);
            if (!out[i].mag) return c->fail(GBR_ENOMEM, "host result allocation");
            if (cof) {   // X / gcd = sign(lc X), 0 / gcd = 0
                gbr_bigpoly &cx = I.dP < 0 ? out_b[i] : out_a[i];
                set_big_int(cx, {{1u, sg}});
                if (!cx.mag) return c->fail(GBR_ENOMEM, "host result allocation");
            }
            continue;
        }
        if (I.dP == 0 || I.dQ == 0) {   // a non-zero constant: gcd of the contents
            set_big_int(out[i], {{I.c, 1}});
            if (!out[i].mag) return c->fail(GBR_ENOMEM, "host result allocation");
            if (cof) {   // each input divided by the integer gcd of the contents
                for (int w = 0; w < 2; ++w) {
                    const int64_t *X = hin + in_off[i] + (w ? p[i].deg + 1 : 0);
                    const int dx = w ? I.dQ : I.dP;
                    std::vector<std::pair<uint64_t, int>> co(dx + 1);
                    for (int t = 0; t <= dx; ++t) {
                        const int64_t v = X[t];
                        const uint64_t mag = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
                        co[t] = {mag / I.c, v == 0 ? 0 : (v < 0 ? -1 : 1)};
                    }
                    gbr_bigpoly &cx = w ? out_b[i] : out_a[i];
                    set_big_int(cx, co);
                    if (!cx.mag) return c->fail(GBR_ENOMEM, "host result allocation");
                }
            }
            continue;
        }
        pending.push_back(i);
    }
    // ---- modular attempts
    const ModP *HM = host_mods();
    const int NP = num_primes();
    int spare = 3;
    std::vector<int> next_prime(n, 0);   // table cursor per job
    while (!pending.empty()) {
        const int m = (int)pending.size();
        std::vector<GcdPlan> plan(n);
        std::vector<int32_t> slotlist;
        int64_t slot_w = 0;
        int maxreg = 1;
        std::vector<int32_t> wl_jobs;
        std::vector<int64_t> wl_start;
        int64_t total = 0;
        for (int ji = 0; ji < m; ++ji) {
            int i = pending[ji];
            const GcdInfo &I = info[i];
            GcdPlan &G = plan[i];
            G.dP = I.dP;
            G.dQ = I.dQ;
            G.cP = I.cP;
            G.cQ = I.cQ;
            G.c = I.c;
            G.b = I.b;
            G.pin_off = in_off[i];
            G.qin_off = in_off[i] + p[i].deg + 1;
            int kneed = primes_for_bits(I.log2B * (1.0 + 1e-9) + 2.0);
            if (kneed < 0) return c->fail(GBR_ELIMIT, "gcd bound needs more than GBR_MAX_PRIMES primes");
            kneed += c->extra_primes;
            G.kcrt = kneed;
            G.slotlist_off = (int64_t)slotlist.size();
            int got = 0;
            int cur = next_prime[i];
            uint64_t alp = I.lcP < 0 ? 0ull - (uint64_t)I.lcP : (uint64_t)I.lcP;
            uint64_t alq = I.lcQ < 0 ? 0ull - (uint64_t)I.lcQ : (uint64_t)I.lcQ;
            while (got < kneed + spare && cur < NP) {
                uint32_t pr = HM[cur].p;
                if (alp % pr != 0 && alq % pr != 0) {   // p must not divide lc(P) lc(Q)
                    slotlist.push_back(cur);
                    ++got;
                }
                ++cur;
            }
            if (got < kneed) return c->fail(GBR_EVERIFY, "ran out of primes for a gcd");
            next_prime[i] = cur;
            G.nslots = got;
            G.S = (std::min(G.dP, G.dQ) + 1) + (G.dP + 1) + (G.dQ + 1);
            G.slot_off = slot_w;
            slot_w += (int64_t)got * G.S;
            maxreg = std::max(maxreg, std::max(G.dP, G.dQ) + 1);
            wl_jobs.push_back(i);
            wl_start.push_back(total);
            total += got;
        }
        wl_start.push_back(total);
        // device buffers for this attempt
        Bufs ab{c, {}};
        GcdPlan *d_plan = (GcdPlan *)ab.get(sizeof(GcdPlan) * n);
        int32_t *d_slotlist = (int32_t *)ab.get(slotlist.size() * 4);
        int32_t *d_sdeg = (int32_t *)ab.get(slotlist.size() * 4);
        uint32_t *d_slots = (uint32_t *)ab.get((size_t)slot_w * 4);
        int64_t *d_wls = (int64_t *)ab.get(wl_start.size() * 8);
        int32_t *d_wlj = (int32_t *)ab.get(wl_jobs.size() * 4);
        if (!d_plan || !d_slotlist || !d_sdeg || !d_slots || !d_wls || !d_wlj)
            return c->fail(GBR_ENOMEM, "device budget too small for the gcd batch");
        e = gcd_copy(c, d_plan, plan.data(), sizeof(GcdPlan) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = gcd_copy(c, d_slotlist, slotlist.data(), slotlist.size() * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = gcd_copy(c, d_wls, wl_start.data(), wl_start.size() * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = gcd_copy(c, d_wlj, wl_jobs.data(), wl_jobs.size() * 4, cudaMemcpyHostToDevice, s);
        L.plan = d_plan;
        L.slots = d_slots;
        L.slotlist = d_slotlist;
        L.sdeg = d_sdeg;
        size_t per_warp = (size_t)2 * maxreg * 4;
        int nw = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp));
        size_t smem = per_warp * nw;
        if (smem > (size_t)kMaxDynSmem) return c->fail(GBR_ELIMIT, "gcd degree too large for shared memory");
        if (e == cudaSuccess) {
            int grid = grid_for((const void *)k_gcd_modp, nw * 32, smem, (total + nw - 1) / nw);
            k_gcd_modp<<<grid, nw * 32, smem, s>>>(L, d_wls, d_wlj, (int)wl_jobs.size(), total, maxreg);
            c->gcd_kernels++;
            c->gcd_subproblems += total;
            e = cudaGetLastError();
        }
        std::vector<int32_t> sdeg(slotlist.size());
        if (e == cudaSuccess) e = gcd_copy(c, sdeg.data(), d_sdeg, sdeg.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "gcd modular stage", e);
        // ---- keep the primes of minimal gcd degree
        std::vector<int32_t> crtlist;
        std::vector<int> ready, retry;
        int64_t garner_w = 0, lift_w = 0, lsign_b = 0, out_w = 0, osign_b = 0, cof_w = 0, cofsign_b = 0;
        int maxL = 1;
        std::vector<int32_t> cj;
        std::vector<int64_t> cs;
        int64_t ctotal = 0;
        for (int ji = 0; ji < m; ++ji) {
            int i = pending[ji];
            GcdPlan &G = plan[i];
            int dmin = INT32_MAX;
            for (int sl = 0; sl < G.nslots; ++sl) dmin = std::min(dmin, sdeg[G.slotlist_off + sl]);
            std::vector<int> good;
            for (int sl = 0; sl < G.nslots && (int)good.size() < G.kcrt; ++sl)
                if (sdeg[G.slotlist_off + sl] == dmin) good.push_back(sl);
            if ((int)good.size() < G.kcrt) {
                retry.push_back(i);
                continue;
            }
            G.dstar = dmin;
            G.crtlist_off = (int64_t)crtlist.size();
            double l2m = 0;
            for (int sl : good) {
                crtlist.push_back(sl);
                l2m += std::log2((double)HM[slotlist[G.slotlist_off + sl]].p);
            }
            G.log2M = l2m;
            G.garner_off = garner_w;
            garner_w += G.kcrt + (int64_t)G.kcrt * (G.kcrt - 1) / 2;
            G.Lcrt = (31 * G.kcrt + 31) / 32;
            G.Lout = G.Lcrt + 2;
            G.Lcof = G.Lcrt + 2;
            G.cof_off = cof_w;
            G.cofsign_off = cofsign_b;
            if (cof) {
                cof_w += (int64_t)((G.dP - dmin + 1) + (G.dQ - dmin + 1)) * G.Lcof;
                cofsign_b += (G.dP - dmin + 1) + (G.dQ - dmin + 1);
            }
            int ncoef = (dmin + 1) + (G.dP - dmin + 1) + (G.dQ - dmin + 1);
            G.lift_off = lift_w;
            lift_w += (int64_t)ncoef * G.Lcrt;
            G.lsign_off = lsign_b;
            lsign_b += ncoef;
            G.out_off = out_w;
            out_w += (int64_t)(dmin + 1) * G.Lout;
            G.osign_off = osign_b;
            osign_b += dmin + 1;
            maxL = std::max(maxL, G.Lcrt);
            ready.push_back(i);
            cj.push_back(i);
            cs.push_back(ctotal);
            ctotal += ncoef;
        }
        cs.push_back(ctotal);
        if (!ready.empty()) {
            Bufs cb{c, {}};
            int32_t *d_crtlist = (int32_t *)cb.get(crtlist.size() * 4);
            uint32_t *d_garner = (uint32_t *)cb.get((size_t)garner_w * 4);
            uint32_t *d_lift = (uint32_t *)cb.get((size_t)lift_w * 4);
            int8_t *d_lsign = (int8_t *)cb.get((size_t)lsign_b);
            uint32_t *d_out = (uint32_t *)cb.get((size_t)out_w * 4);
            int8_t *d_osign = (int8_t *)cb.get((size_t)osign_b);
            int32_t *d_odeg = (int32_t *)cb.get((size_t)n * 4);
            int32_t *d_status = (int32_t *)cb.get((size_t)n * 4);
            uint32_t *d_cof = cof ? (uint32_t *)cb.get((size_t)cof_w * 4) : nullptr;
            int8_t *d_cofsign = cof ? (int8_t *)cb.get((size_t)cofsign_b) : nullptr;
            if (cof && (!d_cof || !d_cofsign)) return c->fail(GBR_ENOMEM, "device budget too small for the gcd cofactors");
            int32_t *d_ready = (int32_t *)cb.get(ready.size() * 4);
            int64_t *d_cs = (int64_t *)cb.get(cs.size() * 8);
            int32_t *d_cj = (int32_t *)cb.get(cj.size() * 4);
            if (!d_crtlist || !d_garner || !d_lift || !d_lsign || !d_out || !d_osign || !d_odeg || !d_status ||
                !d_ready || !d_cs || !d_cj)
                return c->fail(GBR_ENOMEM, "device budget too small for the gcd lift");
            e = gcd_copy(c, d_plan, plan.data(), sizeof(GcdPlan) * n, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = gcd_copy(c, d_crtlist, crtlist.data(), crtlist.size() * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = gcd_copy(c, d_ready, ready.data(), ready.size() * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = gcd_copy(c, d_cs, cs.data(), cs.size() * 8, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = gcd_copy(c, d_cj, cj.data(), cj.size() * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, (size_t)n * 4, s);
            L.crtlist = d_crtlist;
            L.garner = d_garner;
            L.lift = d_lift;
            L.lsign = d_lsign;
            L.out = d_out;
            L.osign = d_osign;
            L.odeg = d_odeg;
            L.cof = d_cof;
            L.cofsign = d_cofsign;
            L.status = d_status;
            const int nr = (int)ready.size();
            if (e == cudaSuccess) {
                int64_t it = (int64_t)nr * GBR_MAX_PRIMES;
                int grid = (int)std::min<int64_t>((it + 255) / 256, 4096);
                k_gcd_garner<<<grid, 256, 0, s>>>(L, d_ready, nr);
                c->gcd_kernels++;
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                // one thread per coefficient, no warp-wide operation: blocks below a
                // warp are fine for very wide lifts
                int block = 128;
                while (block > 1 && (size_t)maxL * block * 4 > 160 * 1024) block >>= 1;
                size_t sm2 = (size_t)maxL * block * 4;
                if (sm2 > (size_t)kMaxDynSmem) e = cudaErrorInvalidValue;
                if (e == cudaSuccess) {
                    int grid = grid_for((const void *)k_gcd_crt, block, sm2, (ctotal + block - 1) / block);
                    k_gcd_crt<<<grid, block, sm2, s>>>(L, d_cs, d_cj, (int)cj.size(), ctotal, maxL);
                    c->gcd_kernels++;
                    e = cudaGetLastError();
                }
            }
            if (e == cudaSuccess) {
                k_gcd_check<<<(nr * 32 + 127) / 128, 128, 0, s>>>(L, d_ready, nr);
                c->gcd_kernels++;
                e = cudaGetLastError();
            }
            std::vector<int32_t> st(n), od(n);
            std::vector<uint32_t> hout((size_t)out_w);
            std::vector<int8_t> hos((size_t)osign_b);
            int32_t herr = 0;
            if (e == cudaSuccess) e = gcd_copy(c, st.data(), d_status, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = gcd_copy(c, od.data(), d_odeg, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && out_w) e = gcd_copy(c, hout.data(), d_out, (size_t)out_w * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && osign_b) e = gcd_copy(c, hos.data(), d_osign, (size_t)osign_b, cudaMemcpyDeviceToHost, s);
            std::vector<uint32_t> hcof(cof ? (size_t)cof_w : 0);
            std::vector<int8_t> hcs(cof ? (size_t)cofsign_b : 0);
            if (e == cudaSuccess && cof && cof_w) e = gcd_copy(c, hcof.data(), d_cof, (size_t)cof_w * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && cof && cofsign_b) e = gcd_copy(c, hcs.data(), d_cofsign, (size_t)cofsign_b, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = gcd_copy(c, &herr, c->d_err, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "gcd lift and check", e);
            if (herr) return c->fail(GBR_EDEVICE, "gcd device-side consistency check failed");
            // the results verified in this attempt share one host block
            std::vector<int> done;
            for (int i : ready) {
                if (st[i] != 1) retry.push_back(i);
                else done.push_back(i);
            }
            // per done job: the gcd, then (when asked for) the two cofactors
            const int per = cof ? 3 : 1;
            std::vector<gbr_bigpoly> tmp(done.size() * per);
            for (size_t t = 0; t < done.size(); ++t) {
                const GcdPlan &G = plan[done[t]];
                tmp[t * per].deg = od[done[t]];
                tmp[t * per].limbs = G.Lout;
                if (cof) {
                    tmp[t * per + 1].deg = G.dP - od[done[t]];
                    tmp[t * per + 1].limbs = G.Lcof;
                    tmp[t * per + 2].deg = G.dQ - od[done[t]];
                    tmp[t * per + 2].limbs = G.Lcof;
                }
            }
            if (!tmp.empty() && !gbr_alloc_results(tmp.data(), (int)tmp.size()))
                return c->fail(GBR_ENOMEM, "host result allocation");
            for (size_t t = 0; t < done.size(); ++t) {
                const int i = done[t];
                const GcdPlan &G = plan[i];
                out[i] = tmp[t * per];
                if (out[i].deg >= 0) {
                    std::memcpy(out[i].mag, hout.data() + G.out_off, (size_t)(out[i].deg + 1) * G.Lout * 4);
                    std::memcpy(out[i].sign, hos.data() + G.osign_off, (size_t)out[i].deg + 1);
                }
                if (cof) {
                    out_a[i] = tmp[t * per + 1];
                    out_b[i] = tmp[t * per + 2];
                    const int na = out_a[i].deg + 1, nb = out_b[i].deg + 1;
                    std::memcpy(out_a[i].mag, hcof.data() + G.cof_off, (size_t)na * G.Lcof * 4);
                    std::memcpy(out_a[i].sign, hcs.data() + G.cofsign_off, (size_t)na);
                    std::memcpy(out_b[i].mag, hcof.data() + G.cof_off + (int64_t)na * G.Lcof, (size_t)nb * G.Lcof * 4);
                    std::memcpy(out_b[i].sign, hcs.data() + G.cofsign_off + na, (size_t)nb);
                }
            }
        }
        pending = retry;
        spare = spare * 4 + 8;
        if (spare > GBR_MAX_PRIMES) spare = GBR_MAX_PRIMES;
        for (int i : retry)
            if (next_prime[i] >= NP) return c->fail(GBR_EVERIFY, "gcd check failed with every table prime");
    }
    return GBR_OK;
}

int gbr_gcd_cof_locked(gbr_ctx *c, int n, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *out,
                       gbr_bigpoly *out_a, gbr_bigpoly *out_b) {
    NvtxScope call("gbr: gcd batch");
    int st;
    const auto t0 = std::chrono::steady_clock::now();
    if (c->stats_on) cudaEventRecord(c->ev[0], c->stream);
    try {
        st = gcd_batch_locked(c, n, p, q, out, out_a, out_b);
        if (c->stats_on) {
            // the whole call on the context's stream: copies, kernels and the host
            // planning between them (the gcd path synchronises after each stage)
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
    if (st != GBR_OK)
        for (int i = 0; i < n; ++i) {
            gbr_free_result(c, &out[i]);
            if (out_a) gbr_free_result(c, &out_a[i]);
            if (out_b) gbr_free_result(c, &out_b[i]);
        }
    return st;
}

extern "C" int gbr_gcd_batch(gbr_ctx *c, int n, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *out) {
    if (!c || n < 0 || (n && (!p || !q || !out))) return GBR_EINVAL;
    if (n == 0) return GBR_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return gbr_gcd_cof_locked(c, n, p, q, out, nullptr, nullptr);
}

extern "C" int gbr_gcd_cofactors_batch(gbr_ctx *c, int n, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *g,
                                       gbr_bigpoly *p_over_g, gbr_bigpoly *q_over_g) {
    if (!c || n < 0 || (n && (!p || !q || !g || !p_over_g || !q_over_g))) return GBR_EINVAL;
    if (n == 0) return GBR_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return gbr_gcd_cof_locked(c, n, p, q, g, p_over_g, q_over_g);
}

extern "C" int gbr_gcd(gbr_ctx *c, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *out) {
    if (!p || !q) return GBR_EINVAL;
    return gbr_gcd_batch(c, 1, p, q, out);
}
