// Device stages of the multi-modular resultant res_var(f, g) in Z[x].
//
// The scheme is the divide-conquer-combine method the paper's Section 4
// ("Symbolic Speedups") describes after Brown and Collins: (1) modular and
// evaluation homomorphisms turn the bivariate problem into independent
// subproblems over prime fields, (2) each subproblem is solved on its own,
// (3) interpolation in x and Chinese remaindering recover the integer result.
// Stages:
//   bounds   (A0) actual degrees and the Hadamard bound, one warp per pair
//   reduce   (A1) coefficients -> residues mod every prime (Montgomery form), one
//            thread per (pair, coefficient slot, run of 32 primes)
//   evalres  (A2+A3) one thread per (pair, prime, point): Horner evaluation of
//            every y-coefficient at x = point, then the univariate resultant with
//            formal degrees by fraction-free remainder steps
//   interp   (A4) one warp per (pair, prime): Newton interpolation on the
//            points 0..P-1 and conversion to monomial coefficients
//   crt      (A5) one thread per (pair, coefficient) on up to 64 primes (one warp per
//            coefficient up to 512): Garner mixed-radix digits, symmetric lift,
//            magnitude limbs
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "gbr_device.cuh"

namespace gbr {

// ------------------------------------------------------------------ A0: bounds

// Top bit e and the top 32 bits of |c| (plus one when any lower bit is set; at
// most 2^32 - 1 + 1, kept as 2^31 with e + 1 then) of a two's-complement
// multi-word integer, so that |c| <= m32 2^(e - 31); false for zero.
__device__ bool coef_top_bits(const uint64_t *w, int W, int &e, uint32_t &m32) {
    uint64_t mag[8];
    const bool neg = (int64_t)w[W - 1] < 0;
    uint64_t carry = 1;
    for (int i = 0; i < W; ++i) {
        uint64_t v = w[i];
        if (neg) {
            v = ~v + carry;
            carry = (carry && v == 0) ? 1 : 0;
        }
        mag[i] = v;
    }
    int t = W - 1;
    while (t >= 0 && mag[t] == 0) --t;
    if (t < 0) return false;
    const int lz = __clzll((long long)mag[t]);
    e = 64 * t + 63 - lz;
    // the 64 bits from the top bit down, and whether anything below them is set
    uint64_t top = mag[t] << lz;
    bool rest = false;
    if (t > 0) {
        if (lz) top |= mag[t - 1] >> (64 - lz);
        rest = (mag[t - 1] << lz) != 0;
        for (int i = t - 2; i >= 0 && !rest; --i) rest = mag[i] != 0;
    }
    m32 = (uint32_t)(top >> 32);
    rest = rest || (uint32_t)top != 0;
    if (rest) {
        if (m32 == 0xFFFFFFFFu) {
            m32 = 0x80000000u;
            ++e;
        } else {
            ++m32;
        }
    }
    return true;
}

__device__ __forceinline__ const uint64_t *coef_ptr(const uint64_t *coef, const PolyDesc &d, int r, int c) {
    return coef + d.off + ((int64_t)r * d.rstride + (int64_t)c * d.cstride) * d.words;
}

// Scans one polynomial row by row (one warp per pair): row degrees, log2 of the
// row 1-norms, degrees.  For disc, g = d f / d var is formed on the fly:
// g_r = (r+1) f_{r+1}.  The row norms are kept in shared memory; the warp
// evaluates the scaled Hadamard bound for every lambda in single precision with
// directed rounding and explicit error margins (each value is an upper bound)
// and keeps the smallest (the FP64 pipe of this part is slow).
constexpr int kBoundsWarps = 4;
constexpr int kBoundsTeamPairs = 256;   // batches up to this size: four warps per pair

// Row quantity of the Hadamard bound.  For a row f_r(x) = sum_a c_a x^a with
// int64 coefficients: G = A_0 + 2 sum_{k>0} |A_k|, A_k = sum_a c_a c_{a+k} (the
// autocorrelation), which bounds |f_r(x)|^2 on |x| = 1 because
// |f_r(x)|^2 = A_0 + 2 sum_k A_k cos(k theta); it never exceeds the squared
// 1-norm and is far smaller when the signs cancel.  The row is staged in shared
// memory.  Coefficients of 2^56 and more: double sums with the error term
// gamma sum |c_a c_{a+k}|, gamma = 2 (L+1) 2^-53 (covering the conversions,
// products and the sum of L terms), so G stays an upper bound.  Wider
// coefficients, and rows longer than kRowBuf (where the O(L^2) sums would
// dominate the whole run): log2 of the 1-norm by a log-sum-exp over the
// coefficients' log2 magnitudes (G <= 1-norm^2, so still an upper bound).
constexpr int kRowBuf = 128;   // coefficients of one row staged per warp

// log2 of a positive 128-bit integer hi 2^64 + lo, rounded up to a float: the
// top 32 bits (plus one when lower bits are set) as a float rounded up, log2f of
// it (in [31, 32], within 1 ulp < 2^-19, covered by adding 2^-18), plus the shift
__device__ __forceinline__ float log2_up_u128(uint64_t hi, uint64_t lo) {
    const unsigned __int128 G = ((unsigned __int128)hi << 64) | lo;
    const int e = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    uint32_t m32;
    bool rest = false;
    int s = 0;
    if (e >= 31) {
        s = e - 31;
        m32 = (uint32_t)(G >> s);
        rest = s > 0 && (G << (128 - s)) != 0;
    } else {
        m32 = (uint32_t)(lo << (31 - e));
        s = e - 31;
    }
    float mf = __uint2float_ru(m32);
    if (rest) mf = __fadd_ru(mf, 1.0f);
    return __fadd_ru((float)s, __fadd_ru(log2f(mf), 0x1p-18f));
}

// log2 x rounded up to a float, for a positive finite double x: the exponent
// from the bits, log2f of the mantissa in [1, 2) (converted upward; log2f is
// within 1 ulp, below 2^-23 there, covered by the 2^-20 added), the sum rounded up
__device__ __forceinline__ float log2_up(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const double mant = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    return __fadd_ru((float)e, __fadd_ru(log2f(__double2float_ru(mant)), 0x1p-20f));
}

__device__ float row_l1_log2_up(const uint64_t *coef, const PolyDesc &P, int r, int lane, int &cmax);

// An upper bound of log2 of the row norm used by the Hadamard bound, as a float
// (-inf for a zero row).  Single-word rows of at most kRowBuf coefficients: half
// the log2 of the autocorrelation quantity G; with every |c| < 2^56, G is summed
// exactly (int64 terms below 2^27, else 128-bit products; G < 2^127) and its log2
// taken from its leading bits; wider single-word coefficients use the double sum
// with its error term.  Multi-word rows and longer rows: the log2 of the 1-norm by
// a log-sum-exp, rounded up.
__device__ float row_log2_up(const uint64_t *coef, const PolyDesc &P, int r, int lane, int &cmax, int64_t *rb) {
    cmax = -1;
    if (P.words == 1) {
        uint64_t big = 0;   // OR of the |c|
        for (int c = lane; c <= P.cols; c += 32) {
            const int64_t v = (int64_t)coef_ptr(coef, P, r, c)[0];
            if (c < kRowBuf) rb[c] = v;
            if (v) cmax = c;
            big |= v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
        }
        for (int o = 16; o; o >>= 1) {
            cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
            big |= __shfl_xor_sync(0xffffffffu, big, o);
        }
        __syncwarp();
        if (cmax < 0) return -INFINITY;
        const int L = cmax + 1;
        if (L > kRowBuf) return row_l1_log2_up(coef, P, r, lane, cmax);
        if (big < (1ull << 56)) {
            // exact: |A_k| < 128 * 2^112, G < 2^127
            unsigned __int128 acc = 0;
            for (int k = lane; k < L; k += 32) {
                unsigned __int128 ak;
                if (big < (1ull << 27)) {
                    int64_t sk = 0;
                    for (int a = 0; a + k < L; ++a) sk += rb[a] * rb[a + k];
                    ak = (unsigned __int128)(uint64_t)(sk < 0 ? -sk : sk);
                } else {
                    __int128 sk = 0;
                    for (int a = 0; a + k < L; ++a) sk += (__int128)rb[a] * rb[a + k];
                    ak = (unsigned __int128)(sk < 0 ? -sk : sk);
                }
                acc += ak << (k ? 1 : 0);
            }
            uint64_t lo = (uint64_t)acc, hi = (uint64_t)(acc >> 64);
            for (int o = 16; o; o >>= 1) {
                const uint64_t olo = __shfl_xor_sync(0xffffffffu, lo, o), ohi = __shfl_xor_sync(0xffffffffu, hi, o);
                lo += olo;
                hi += ohi + (lo < olo ? 1u : 0u);
            }
            __syncwarp();
            return 0.5f * log2_up_u128(hi, lo);
        }
        double G = 0.0;
        const double gam = 2.0 * (L + 1) * 0x1p-53;
        for (int k = lane; k < L; k += 32) {
            double sk = 0.0, tk = 0.0;
            for (int a = 0; a + k < L; ++a) {
                const double x = (double)rb[a];
                const double y = (double)rb[a + k];
                sk = fma(x, y, sk);
                tk = fma(fabs(x), fabs(y), tk);
            }
            G += (k ? 2.0 : 1.0) * (fabs(sk) + gam * tk);
        }
        for (int o = 16; o; o >>= 1) G += __shfl_xor_sync(0xffffffffu, G, o);
        __syncwarp();
        // G: a lane's sum of about L / 32 <= 4 non-negative terms plus five shuffle
        // additions, so the relative error stays below 2^-43
        return 0.5f * log2_up(G * (1.0 + 0x1p-40));
    }
    return row_l1_log2_up(coef, P, r, lane, cmax);
}

// log2 of the 1-norm of row r, rounded up (-inf for a zero row; cmax gets the
// row's degree).  Each |c| <= m32 2^(e - 31) with m32 its top 32 bits (plus one
// when lower bits are set) and e its top bit; the terms are summed in float
// relative to the row's largest e, rounded up (terms below 2^-100 of it are
// raised to 2^-100, which only enlarges the sum).
__device__ float row_l1_log2_up(const uint64_t *coef, const PolyDesc &P, int r, int lane, int &cmax) {
    cmax = -1;
    int emax = -1;
    for (int c = lane; c <= P.cols; c += 32) {
        int e;
        uint32_t m32;
        if (coef_top_bits(coef_ptr(coef, P, r, c), P.words, e, m32)) {
            cmax = c;
            emax = max(emax, e);
        }
    }
    for (int o = 16; o; o >>= 1) {
        cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    if (cmax < 0) return -INFINITY;
    float sum = 0.0f;
    for (int c = lane; c <= P.cols; c += 32) {
        int e;
        uint32_t m32;
        if (coef_top_bits(coef_ptr(coef, P, r, c), P.words, e, m32)) {
            const float t = __uint2float_ru(m32) * 0x1p-31f;   // in [1, 2], exact scaling
            sum = __fadd_ru(sum, e - emax < -100 ? 0x1p-100f : ldexpf(t, e - emax));
        }
    }
    for (int o = 16; o; o >>= 1) sum = __fadd_ru(sum, __shfl_xor_sync(0xffffffffu, sum, o));
    // sum in [1, 2^15) (at most 16384 terms of at most 2): log2f within 1 ulp
    // (at most 2^-20 below 16), covered by 2^-19
    return __fadd_ru((float)emax, __fadd_ru(log2f(sum), 0x1p-19f));
}

// ceil(x 2^16) for a finite |x| < 2^15 (the scaling is exact)
__device__ __forceinline__ long long fx16_up(float x) { return (long long)__float2int_ru(x * 65536.0f); }

// 2 tm + log2 s, in units of 2^-16 and rounded up, for the sum s of the terms
// exp2f(max(2 (t_k - tm) rounded up, -120)) of a set of exponents t_k with the
// finite maximum tm (or any tm at least as large whose largest term is at least
// 2^-100): an upper bound of log2 sum_k 2^(2 t_k).  exp2f (within 2
// ulp) and the round-up sums of at most 256 terms are covered by the factor
// 1 + 2^-20, log2f of s in [2^-100, 2^9) (within 1 ulp, at most 2^-17 there) by
// adding 2^-14;
// terms below 2^-120 of the largest are raised to it (that only enlarges it).
__device__ __forceinline__ long long log2_sum_fx(float tm, float s) {
    return 2 * fx16_up(tm) + fx16_up(__fadd_ru(log2f(__fmul_ru(s, 1.0f + 0x1p-20f)), 0x1p-14f));
}

__device__ __forceinline__ float exp2_term(float t, float tm) { return exp2f(fmaxf(2.0f * __fsub_ru(t, tm), -120.0f)); }

// Twice (the log2 of the scaled Hadamard bound's smaller form minus m n l2lam),
// in units of 2^-16 and rounded up, evaluated warp-parallel: lanes split the rows
// for the scaled squared norms and the columns for their logarithms.  lf, lg are
// float upper bounds of the log2 row norms (-inf for zero rows); the scaled
// exponents t = lf_i + i l2lam are rounded up; the row sums are shifted by their
// own largest term (the rows of f, the rows of g), a column by the overall
// largest term M unless its own is more than 50 below M (then by its own); the outer
// sums are exact integer sums.  LLONG_MIN when a column of the Sylvester matrix
// is zero (the resultant vanishes).  l2lam is a multiple of 1/4 in [-2^2, 2^3].
__device__ long long scaled_hadamard_fx(const float *lf, int m, const float *lg, int n, float l2lam, float *tf,
                                        float *tg, float *ef, float *eg, int lane) {
    float Mf = -INFINITY, Mg = -INFINITY;
    for (int i = lane; i <= m; i += 32) {
        const float t = lf[i] == -INFINITY ? -INFINITY : __fmaf_ru((float)i, l2lam, lf[i]);
        tf[i] = t;
        Mf = fmaxf(Mf, t);
    }
    for (int j = lane; j <= n; j += 32) {
        const float t = lg[j] == -INFINITY ? -INFINITY : __fmaf_ru((float)j, l2lam, lg[j]);
        tg[j] = t;
        Mg = fmaxf(Mg, t);
    }
    for (int o = 16; o; o >>= 1) {
        Mf = fmaxf(Mf, __shfl_xor_sync(0xffffffffu, Mf, o));
        Mg = fmaxf(Mg, __shfl_xor_sync(0xffffffffu, Mg, o));
    }
    __syncwarp();
    // the terms once more against the overall maximum M, for the columns
    const float M = fmaxf(Mf, Mg);
    float sf = 0.0f, sg = 0.0f;
    for (int i = lane; i <= m; i += 32) {
        const bool z = tf[i] == -INFINITY;
        if (!z) sf = __fadd_ru(sf, exp2_term(tf[i], Mf));
        ef[i] = z ? 0.0f : exp2_term(tf[i], M);
    }
    for (int j = lane; j <= n; j += 32) {
        const bool z = tg[j] == -INFINITY;
        if (!z) sg = __fadd_ru(sg, exp2_term(tg[j], Mg));
        eg[j] = z ? 0.0f : exp2_term(tg[j], M);
    }
    for (int o = 16; o; o >>= 1) {
        sf = __fadd_ru(sf, __shfl_xor_sync(0xffffffffu, sf, o));
        sg = __fadd_ru(sg, __shfl_xor_sync(0xffffffffu, sg, o));
    }
    long long row = 0;
    if (n > 0) row += (long long)n * log2_sum_fx(Mf, sf);
    if (m > 0) row += (long long)m * log2_sum_fx(Mg, sg);
    long long col = 0;
    int zero = 0;
    for (int c = lane; c < m + n; c += 32) {
        // f rows r = 0..n-1 hold f_{m-(c-r)} in column c; g rows r = 0..m-1 hold g_{n-(c-r)}
        const int fr0 = c - m > 0 ? c - m : 0, fr1 = c < n - 1 ? c : n - 1;
        const int gr0 = c - n > 0 ? c - n : 0, gr1 = c < m - 1 ? c : m - 1;
        float mc = -INFINITY;
        for (int r = fr0; r <= fr1; ++r) mc = fmaxf(mc, tf[m - (c - r)]);
        for (int r = gr0; r <= gr1; ++r) mc = fmaxf(mc, tg[n - (c - r)]);
        if (mc == -INFINITY) {
            zero = 1;
            continue;
        }
        float sc = 0.0f;
        if (mc >= M - 50.0f) {
            // the terms against M: the largest is at least 2^-100, so raising the
            // others to 2^-120 enlarges the sum by at most 256 2^-20 of it
            for (int r = fr0; r <= fr1; ++r) sc = __fadd_ru(sc, ef[m - (c - r)]);
            for (int r = gr0; r <= gr1; ++r) sc = __fadd_ru(sc, eg[n - (c - r)]);
            col += log2_sum_fx(M, sc);
        } else {
            for (int r = fr0; r <= fr1; ++r)
                if (tf[m - (c - r)] != -INFINITY) sc = __fadd_ru(sc, exp2_term(tf[m - (c - r)], mc));
            for (int r = gr0; r <= gr1; ++r)
                if (tg[n - (c - r)] != -INFINITY) sc = __fadd_ru(sc, exp2_term(tg[n - (c - r)], mc));
            col += log2_sum_fx(mc, sc);
        }
    }
    for (int o = 16; o; o >>= 1) col += __shfl_xor_sync(0xffffffffu, col, o);
    zero = __any_sync(0xffffffffu, zero);
    if (zero) return LLONG_MIN;
    const long long lam = (long long)m * n * (long long)__float2int_rn(l2lam * 131072.0f);   // 2 m n l2lam 2^16
    return (row < col ? row : col) - lam;
}

// Degree statistics of one polynomial from the row degrees rd[0..rows] (-1: zero row),
// warp-parallel over the rows: the degree, the largest x-degree, the total degree, the
// coefficient count up to the degree, the leading row's x-degree.
__device__ void row_stats(const int32_t *rd, int rows, int lane, int &mdeg, int &dxmax, int &td, int &terms_upto,
                          int &lcd) {
    int md = -1, dx = -1, t = -1;
    for (int r = lane; r <= rows; r += 32) {
        const int c = rd[r];
        if (c >= 0) {
            md = max(md, r);
            dx = max(dx, c);
            t = max(t, r + c);
        }
    }
    for (int o = 16; o; o >>= 1) {
        md = max(md, __shfl_xor_sync(0xffffffffu, md, o));
        dx = max(dx, __shfl_xor_sync(0xffffffffu, dx, o));
        t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
    }
    int terms = 0;
    for (int r = lane; r <= md; r += 32) terms += rd[r] + 1;
    for (int o = 16; o; o >>= 1) terms += __shfl_xor_sync(0xffffffffu, terms, o);
    mdeg = md;
    dxmax = dx;
    td = t;
    terms_upto = md >= 0 ? terms : 0;
    lcd = md >= 0 ? rd[md] : -1;
}

// One warp per pair (four pairs per block), or, for batches of at most
// kBoundsTeamPairs pairs, four warps per pair (a block per pair: the rows and the
// scalings lambda split over the warps, the row statistics taken from the row degrees
// afterwards, the smallest bound over the warps): the same quantities either way, the
// team only shortens a small batch's latency.
// (at most 72 registers: seven 4-warp blocks per SM, so a batch of 4096 pairs
// runs in one wave on 152 SMs)
__global__ void __launch_bounds__(kBoundsWarps * 32, 7) k_bounds(ResLaunch L, int team) {
    __shared__ float lff[kBoundsWarps][GBR_MAX_YDEG + 2], lgf[kBoundsWarps][GBR_MAX_YDEG + 2];
    __shared__ float tbuf[kBoundsWarps][2][GBR_MAX_YDEG + 2];
    __shared__ float xbuf[kBoundsWarps][2][GBR_MAX_YDEG + 2];
    __shared__ int64_t rbuf[kBoundsWarps][kRowBuf];
    __shared__ long long tbest[kBoundsWarps];
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // team: warp wt of T = kBoundsWarps shares pair blockIdx.x; else T = 1, wt = 0
    const int T = team ? kBoundsWarps : 1, wt = team ? wib : 0, slot = team ? 0 : wib;
    const int warp = team ? blockIdx.x : (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= L.npairs) return;   // (a team's block is never past the end: the grid is the batch)
    const PairDesc D = L.desc[warp];
    PairBound B;
    B.tg = 0;
    B.lcdg = -1;
    B.pad = 0;
    for (int which = 0; which < 2; ++which) {
        if (which == 1 && D.disc) break;
        const PolyDesc &P = which ? D.g : D.f;
        float *ln_out = which ? lgf[slot] : lff[slot];
        int mdeg = -1, dxmax = -1, td = -1, terms = 0, terms_upto = 0, lcd = -1;
        int mdeg_g = -1, dx_g = -1, td_g = -1, terms_g = 0, terms_g_upto = 0, lcd_g = -1;
        for (int r = wt; r <= P.rows; r += T) {
            int cmax;
            const float ln = row_log2_up(L.coef, P, r, lane, cmax, rbuf[wib]);
            if (lane == 0) {
                L.rowdeg[P.rowdeg_off + r] = cmax;
                if (r <= GBR_MAX_YDEG) ln_out[r] = ln;
            }
            terms += cmax + 1;
            if (cmax >= 0) {
                mdeg = r;
                lcd = cmax;
                terms_upto = terms;
                dxmax = max(dxmax, cmax);
                td = max(td, r + cmax);
            }
            if (which == 0 && D.disc && r >= 1) {
                // row r - 1 of d f / d var is r f_r: its norm is r times f_r's
                if (lane == 0) {
                    L.rowdeg[D.g.rowdeg_off + r - 1] = cmax;
                    if (r - 1 <= GBR_MAX_YDEG)
                        lgf[slot][r - 1] =
                            ln == -INFINITY ? -INFINITY : __fadd_ru(ln, __fadd_ru(log2f((float)r), 0x1p-19f));
                }
                terms_g += cmax + 1;
                if (cmax >= 0) {
                    mdeg_g = r - 1;
                    lcd_g = cmax;
                    terms_g_upto = terms_g;
                    dx_g = max(dx_g, cmax);
                    td_g = max(td_g, r - 1 + cmax);
                }
            }
        }
        if (team) {
            // the rows were split over the warps: the statistics from the row degrees
            // every warp wrote (visible to the block after the barrier)
            __syncthreads();
            row_stats(L.rowdeg + P.rowdeg_off, P.rows, lane, mdeg, dxmax, td, terms_upto, lcd);
            if (which == 0 && D.disc)
                row_stats(L.rowdeg + D.g.rowdeg_off, P.rows - 1, lane, mdeg_g, dx_g, td_g, terms_g_upto, lcd_g);
        }
        __syncwarp();
        if (which == 0) {
            B.m = mdeg; B.dxf = dxmax; B.tdf = td; B.tf = terms_upto; B.lcdf = lcd;
            if (D.disc) {
                B.n = mdeg_g; B.dxg = dx_g; B.tdg = td_g; B.tg = terms_g_upto; B.lcdg = lcd_g;
            }
        } else {
            B.n = mdeg; B.dxg = dxmax; B.tdg = td; B.tg = terms_upto; B.lcdg = lcd;
        }
    }
    __syncwarp();
    double lb = 0.0;
    if (B.m >= 0 && B.n >= 0 && B.m <= GBR_MAX_YDEG && B.n <= GBR_MAX_YDEG && (B.m > 0 || B.n > 0)) {
        // every lambda gives a valid bound; each evaluation is itself an upper bound
        long long best = LLONG_MAX;
        for (int l = wt; l < kBoundLambdas; l += T) {
            const long long v = scaled_hadamard_fx(lff[slot], B.m, lgf[slot], B.n, bound_lambda_f(l), tbuf[wib][0],
                                                   tbuf[wib][1], xbuf[wib][0], xbuf[wib][1], lane);
            best = v < best ? v : best;
        }
        if (team) {
            if (lane == 0) tbest[wib] = best;
            __syncthreads();
            for (int t = 0; t < kBoundsWarps; ++t) best = tbest[t] < best ? tbest[t] : best;
        }
        lb = best == LLONG_MIN ? -INFINITY : (double)best * 0x1p-17 + 0x1p-10;
    } else if (team) {
        __syncthreads();   // (uniform over the block: every warp of the team sees the same B)
    }
    B.log2B = lb;
    if (lane == 0 && wt == 0) L.bounds[warp] = B;
}

// Summed forms of the bound for small shapes (y-degrees at most kSumMaxY, entries of
// x-degree at most kSumMaxX, coefficients below 2^28 in magnitude; one-word inputs).
// For a row or a column of the Sylvester matrix with entries h_e scaled by
// w_e = lambda^(2 deg e), the squared norm at x = e^{it} is C_0 + 2 sum_k C_k cos kt with
// C_k = sum_e w_e A_k(h_e) (A_k the autocorrelation of h_e's x-coefficients), at most
// C_0 + 2 sum_k |C_k|: the absolute values taken after the sum over the entries, never
// more than the per-entry form k_bounds uses.  One warp per pair, after k_bounds: the
// autocorrelations exactly in 64-bit integers (|A_k| < 25 2^56; a lane per entry, the
// entry's coefficients in registers), then one lane per column (and per row form), each
// C_k in single precision with an error term (|C_k| bounded by |computed C_k| + 2^-16
// times the sum of the terms' magnitudes: the conversion of A_k, the rounded weight and
// the at most 50 roundings of the sum stay below 2^-18.3 of it), every further sum
// rounded upward, log2f padded by 2^-13 (its error is 1 ulp), the products over rows and
// columns summed in 2^-17 fixed point; at lambda = 1 and 2^(1/8) (weights 2^(deg / 4),
// from a table rounded to nearest).  The pair's log2 B is lowered when a summed form is
// smaller.
constexpr int kSumMaxY = 24, kSumMaxX = 24, kSumK = kSumMaxX + 1, kSumWarps = 1;
constexpr long long kSumCoefLimit = 1ll << 28;
__constant__ float c_sum_w[kSumMaxY + 1] = {
    1.0f,         1.18920712f,  1.41421356f,  1.68179283f,  2.0f,         2.37841423f,  2.82842712f,
    3.36358566f,  4.0f,         4.75682846f,  5.65685425f,  6.72717132f,  8.0f,         9.51365692f,
    11.3137085f,  13.45434264f, 16.0f,        19.02731384f, 22.627417f,   26.90868529f, 32.0f,
    38.05462768f, 45.254834f,   53.81737058f, 64.0f};   // 2^(d / 4)

__device__ __forceinline__ long long sum_coef(const ResLaunch &L, const PolyDesc &P, int r, int c) {
    return (r <= P.rows && c <= P.cols) ? (long long)coef_ptr(L.coef, P, r, c)[0] : 0ll;
}

// The autocorrelation A_0..A_{kSumK-1} of one entry's x-coefficients (zero past its
// degree) into sA[e][.], exactly in 64-bit integers, then rounded to float.  false when
// a coefficient is out of range.
__device__ __forceinline__ bool sum_autocorr(const ResLaunch &L, const PairDesc &D, int m, int e, float *sAe) {
    const bool gside = e > m;
    const int i = gside ? e - m - 1 : e;
    int c[kSumK];
    bool ok = true;
#pragma unroll
    for (int x = 0; x < kSumK; ++x) {
        long long v;
        if (!gside) v = sum_coef(L, D.f, i, x);
        else if (!D.disc) v = sum_coef(L, D.g, i, x);
        else v = (long long)(i + 1) * sum_coef(L, D.f, i + 1, x);
        ok = ok && v < kSumCoefLimit && v > -kSumCoefLimit;
        c[x] = (int)v;
    }
#pragma unroll
    for (int k = 0; k < kSumK; ++k) {
        long long a = 0;
#pragma unroll
        for (int t = 0; t + k < kSumK; ++t) a += (long long)c[t] * c[t + k];
        sAe[k] = (float)a;
    }
    return ok;
}

__global__ void __launch_bounds__(kSumWarps * 32) k_bounds_summed(ResLaunch L) {
    __shared__ float sA[kSumWarps][2 * (kSumMaxY + 1)][kSumK];
    __shared__ float sw[kSumMaxY + 1];   // the weights, read with a different index per lane
    // prefix (sP, sT) and suffix (sQ, sU) sums of w A_k and w |A_k| over each polynomial's entries
    __shared__ float sP[kSumWarps][2][kSumMaxY + 2][kSumK], sT[kSumWarps][2][kSumMaxY + 2][kSumK];
    __shared__ float sQ[kSumWarps][2][kSumMaxY + 2][kSumK], sU[kSumWarps][2][kSumMaxY + 2][kSumK];
    for (int t = threadIdx.x; t <= kSumMaxY; t += blockDim.x) sw[t] = c_sum_w[t];
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (pair >= L.npairs) return;
    PairBound B = L.bounds[pair];
    const PairDesc D = L.desc[pair];
    const int m = B.m, n = B.n;
    if (m < 0 || n < 0 || m > kSumMaxY || n > kSumMaxY || (m == 0 && n == 0) || B.dxf > kSumMaxX ||
        B.dxg > kSumMaxX || D.f.words != 1 || (!D.disc && D.g.words != 1) || !(B.log2B > -INFINITY))
        return;
    // entries: f_0..f_m (index i), then g_0..g_n (index m + 1 + j); for disc g_j = (j+1) f_{j+1}
    const int ne_all = m + n + 2;
    bool ok = true;
    for (int e = lane; e < ne_all; e += 32) ok = sum_autocorr(L, D, m, e, sA[wib][e]) && ok;
    if (!__all_sync(0xffffffffu, ok)) return;
    __syncwarp();
    const int nforms = m + n + 2;   // columns 0..m+n-1, then f's row form, g's row form
    long long best = LLONG_MAX;
    for (int q8 = 0; q8 <= 1; ++q8) {
        // prefix and suffix sums over each polynomial's entries, per power k (lane = k):
        // sP[0][i][k] = sum_{i' < i} w_i' A_k(f_i'), sQ[0][i][k] = sum_{i' >= i}, sT and sU
        // the same of |A_k|; [1] for g.  A Sylvester column's entries of one polynomial
        // start at its first entry or end at its last (both unless m != n), so C_k is one
        // prefix or one suffix value, within 2^-19.2 of the magnitude sum of its own
        // range (27 roundings at most); an interior range takes a difference of prefixes
        // and the magnitude sums of both.  (A suffix taken as the difference of two
        // prefixes would carry the rounding error of the whole sum, which can exceed a
        // short range's own value by orders of magnitude.)
        __syncwarp();
        if (lane < kSumK) {
            for (int side = 0; side < 2; ++side) {
                const int top = side ? n : m, e0 = side ? m + 1 : 0;
                float p = 0.0f, t = 0.0f;
                sP[wib][side][0][lane] = sT[wib][side][0][lane] = 0.0f;
                for (int i = 0; i <= top; ++i) {
                    const float w = q8 ? sw[i] : 1.0f, a = sA[wib][e0 + i][lane];
                    p = fmaf(w, a, p);
                    t = fmaf(w, fabsf(a), t);
                    sP[wib][side][i + 1][lane] = p;
                    sT[wib][side][i + 1][lane] = t;
                }
                p = t = 0.0f;
                sQ[wib][side][top + 1][lane] = sU[wib][side][top + 1][lane] = 0.0f;
                for (int i = top; i >= 0; --i) {
                    const float w = q8 ? sw[i] : 1.0f, a = sA[wib][e0 + i][lane];
                    p = fmaf(w, a, p);
                    t = fmaf(w, fabsf(a), t);
                    sQ[wib][side][i][lane] = p;
                    sU[wib][side][i][lane] = t;
                }
            }
        }
        __syncwarp();
        // C_k and the magnitude sum that bounds its error, over entries lo..hi of one side
        auto range = [&](int side, int lo, int hi, int top, int k, float &c, float &t) {
            if (lo == 0) {
                c += sP[wib][side][hi + 1][k];
                t += sT[wib][side][hi + 1][k];
            } else if (hi == top) {
                c += sQ[wib][side][lo][k];
                t += sU[wib][side][lo][k];
            } else {
                c += sP[wib][side][hi + 1][k] - sP[wib][side][lo][k];
                t += sT[wib][side][hi + 1][k] + sT[wib][side][lo][k];
            }
        };
        long long row = 0, col = 0;   // 2^-17 fixed point
        for (int base = 0; base < nforms; base += 32) {
            const int fi = base + lane;
            long long mine = 0;
            if (fi < nforms && !(fi == m + n && n == 0) && !(fi == m + n + 1 && m == 0)) {
                // the entries of this form: f_i for i in [ilo, ihi], g_j for j in [jlo, jhi]
                int ilo, ihi, jlo, jhi;
                if (fi < m + n) {
                    // column c: f-row r holds f_{m - (c - r)}, g-row r holds g_{n - (c - r)}
                    const int c = fi;
                    ilo = m - c + max(0, c - m);
                    ihi = m - c + min(n - 1, c);
                    jlo = n - c + max(0, c - n);
                    jhi = n - c + min(m - 1, c);
                } else if (fi == m + n) {
                    ilo = 0, ihi = m, jlo = 0, jhi = -1;
                } else {
                    ilo = 0, ihi = -1, jlo = 0, jhi = n;
                }
                const bool hf = ilo <= ihi, hg = jlo <= jhi;
                float S = 0.0f;
                for (int k = 0; k < kSumK; ++k) {
                    // |C_k| at most |computed| (1 + 2^-22) (the one or two roundings of
                    // joining the pieces) + 2^-17 (the magnitude sums, within 2^-19.2)
                    float c = 0.0f, t = 0.0f;
                    if (hf) range(0, ilo, ihi, m, k, c, t);
                    if (hg) range(1, jlo, jhi, n, k, c, t);
                    float up = __fadd_ru(__fmul_ru(fabsf(c), 1.0f + 0x1p-22f), __fmul_ru(t, 0x1p-17f));
                    if (k) up = __fmul_ru(up, 2.0f);
                    S = __fadd_ru(S, up);
                }
                const float l2 = __fadd_ru(log2f(S), 0x1p-13f);
                mine = __float2ll_ru(l2 * 65536.0f);   // 0.5 log2 in 2^-17 units, upward
                if (fi == m + n) mine *= n;             // n copies of f's row
                else if (fi == m + n + 1) mine *= m;    // m copies of g's
            }
            // sums over the lanes: columns and rows apart (exact integers)
            long long cpart = fi < m + n ? mine : 0, rpart = fi >= m + n ? mine : 0;
            for (int o = 16; o; o >>= 1) {
                cpart += __shfl_xor_sync(0xffffffffu, cpart, o);
                rpart += __shfl_xor_sync(0xffffffffu, rpart, o);
            }
            col += cpart;
            row += rpart;
        }
        // lambda^(-mn) = 2^(-mn q8 / 8), exact in 2^-17 units
        const long long v = (row < col ? row : col) - (long long)m * n * q8 * (131072 / 8);
        best = v < best ? v : best;
    }
    const double nb = (double)best * 0x1p-17 + 0x1p-10;
    if (lane == 0 && nb < B.log2B) L.bounds[pair].log2B = nb;
}

cudaError_t launch_bounds(const ResLaunch &L, cudaStream_t s) {
    if (L.npairs <= 0) return cudaSuccess;
    int threads = kBoundsWarps * 32;
    const int team = L.npairs <= kBoundsTeamPairs;
    int blocks = team ? L.npairs : (L.npairs * 32 + threads - 1) / threads;
    k_bounds<<<blocks, threads, 0, s>>>(L, team);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    threads = kSumWarps * 32;
    blocks = (L.npairs * 32 + threads - 1) / threads;
    k_bounds_summed<<<blocks, threads, 0, s>>>(L);
    return cudaGetLastError();
}

// A replayed step re-measures its bounds and checks, pair by pair, that the plan
// it replays still fits them: the same degrees in both variables, the same number
// of points (the degree bound) and the same number of primes, computed from the
// fresh bound exactly as the host planner does (the smallest k with
// sum_{i<k} log2 p_i > log2 B (1 + 1e-9) + 2 + 1e-6; l2pref[k] is that sum).
// Everything else a plan fixes follows from these, so a plan that passes is exact
// for the new inputs; any pair that fails stops the stages (the host plans again).
__global__ void k_plan_check(const PairBound *bounds, const PairPlan *plan, int n, const double *l2pref, int nprimes,
                             int extra, int32_t *flag) {
    bool bad = false;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const PairBound B = bounds[q];
        const PairPlan &p = plan[q];
        if (p.flags & PLAN_ZERO) {
            bad = bad || (B.m >= 0 && B.n >= 0);
            continue;
        }
        // the plan's points must cover the degree bound (a planned point count may be
        // larger: close counts of a batch are shared)
        if (B.m != p.m || B.n != p.n || max(B.dxf, 0) != p.dxf || max(B.dxg, 0) != p.dxg ||
            (int64_t)degree_bound(B) + 1 > p.P) {
            bad = true;
            continue;
        }
        const double bits = B.log2B * (1.0 + 1e-9) + 2.0 + 1e-6;
        int lo = 1, hi = nprimes + 1;   // first k in [1, nprimes] with l2pref[k] > bits, else nprimes + 1
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (l2pref[mid] > bits) hi = mid;
            else lo = mid + 1;
        }
        bad = bad || lo + extra != p.k;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

cudaError_t launch_plan_check(const PairBound *bounds, const PairPlan *plan, int n, const double *l2pref,
                              int extra, int32_t *flag, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * (int64_t)sm_count());
    k_plan_check<<<grid < 1 ? 1 : grid, 256, 0, s>>>(bounds, plan, n, l2pref, num_primes(), extra, flag);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ A1: modular reduction

// Shoup constants of c -> c R^2 for the first kReduceSmemPrimes table primes: with
// W = R^2 mod p, floor(W 2^32 / p) = (W 2^32 - R^3 mod p) / p is congruent to
// -(R^3 mod p) p^-1 = (R^3 mod p) pinv modulo 2^32, and is below 2^32.
// (The table holds more primes than that: its CRT tables already cover the first
// kCrtFastK.)
constexpr int kReduceSmemPrimes = 64;
static_assert(kReduceSmemPrimes <= kCrtFastK, "the table holds the primes whose constants are staged");

__global__ void k_reduce(ResLaunch L, WorkList w) {
    if (stage_skipped(L)) return;
    __shared__ uint32_t sp[kReduceSmemPrimes], sw[kReduceSmemPrimes], swp[kReduceSmemPrimes];
    for (int t = threadIdx.x; t < kReduceSmemPrimes; t += blockDim.x) {
        const ModP M = L.mods[t];
        sp[t] = M.p;
        sw[t] = M.r2;
        swp[t] = L.r34[t].x * M.pinv;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < w.total; base += stride) {
        // a warp's items are consecutive: one search for its first item, and each
        // lane steps over the pair boundaries after it
        int bi = lane == 0 ? wl_find(w.start, w.n, base) : 0;
        bi = __shfl_sync(0xffffffffu, bi, 0);
        const int64_t item = base + lane;
        if (item >= w.total) continue;
        while (bi + 1 < w.n && item >= w.start[bi + 1]) ++bi;
        const int q = w.pairs[bi];
        const PairPlan &P = L.plan[q];
        const PairDesc &D = L.desc[q];
        // item = chunk S + s: slot s for the primes 32 chunk .. 32 chunk + 31 (results
        // on many primes spread over more threads)
        const int64_t local = item - w.start[bi];
        const int chunk = (int)(local / P.S);
        const int s = (int)(local - (int64_t)chunk * P.S);   // below S < 2^31
        const int rf4 = rows4(P.m), rg4 = rows4(P.n);
        const int nf = (P.dxf + 1) * rf4;
        const PolyDesc *src;
        int row, col, mult = 0, nrows;
        if (s < nf) {
            src = &D.f;
            col = s / rf4;
            row = s - col * rf4;
            nrows = P.m + 1;
        } else {
            const int s2 = s - nf;
            col = s2 / rg4;
            row = s2 - col * rg4;
            nrows = P.n + 1;
            if (D.disc) {
                src = &D.f;
                mult = row + 1;
            } else {
                src = &D.g;
            }
        }
        const int S = P.S, I0 = 32 * chunk, K = min(P.k, I0 + 32);
        uint32_t *dst = L.res + P.res_off + s + (int64_t)I0 * S;
        if (row >= nrows) {                       // padding rows hold zeros
            for (int i = I0; i < K; ++i, dst += S) *dst = 0u;
            continue;
        }
        const uint64_t *cp = coef_ptr(L.coef, *src, mult ? row + 1 : row, col);
        int W = src->words;
        if (W == 1) {
            // |c| = hi 2^32 + lo: c R^2 = redc(hi R^4 + lo R^3); the sum is below
            // 2p 2^32, so the reduction leaves a value below 3p.  With hi = 0 (every
            // coefficient of the warp below 2^32) one product: redc(lo R^3) < 2p.
            const int64_t v = (int64_t)cp[0];
            const bool neg = v < 0;
            const uint64_t av = neg ? 0ull - (uint64_t)v : (uint64_t)v;
            const uint32_t hi = (uint32_t)(av >> 32), lo = (uint32_t)av;
            const bool wide = __any_sync(__activemask(), hi != 0u);
            const int32_t *pm = P.pmap_off < 0 ? nullptr : L.pmap + P.pmap_off;
            if (!wide && !mult && !pm && K <= kReduceSmemPrimes) {
                // one Shoup product lo W - q p with q = floor(lo W' / 2^32): in [0, 2p)
                for (int i = I0; i < K; ++i, dst += S) {
                    const uint32_t p = sp[i];
                    uint32_t r = lo * sw[i] - __umulhi(lo, swp[i]) * p;
                    r = min(r, r - p);
                    *dst = neg ? mp_neg(r, p) : r;
                }
                continue;
            }
            for (int i = I0; i < K; ++i, dst += S) {
                const int pi = pm ? pm[i] : i;
                const ModP M = L.mods[pi];
                const uint2 r34 = L.r34[pi];
                uint32_t r;
                if (wide) {
                    const uint64_t t = (uint64_t)hi * r34.y + (uint64_t)lo * r34.x;
                    const uint32_t m = (uint32_t)t * M.pinv;
                    r = (uint32_t)((t + (uint64_t)m * M.p) >> 32);
                    r = min(r, r - M.p);
                } else {
                    r = mp_redc(lo * r34.x, __umulhi(lo, r34.x), M.p, M.pinv);
                }
                r = min(r, r - M.p);
                if (mult) r = mp_mul(r, mp_to((uint32_t)mult, M), M);
                *dst = neg ? mp_neg(r, M.p) : r;
            }
            continue;
        }
        uint64_t wbuf[8];
        for (int i = 0; i < W; ++i) wbuf[i] = cp[i];
        for (int i = I0; i < K; ++i, dst += S) {
            ModP M = L.mods[prime_of(P, L.pmap, i)];
            uint32_t r = mp_from_words(wbuf, W, M);
            if (mult) r = mp_mul(r, mp_to((uint32_t)mult, M), M);
            *dst = mp_mul(r, M.r2, M);   // c R^2: one reduction per Horner step
        }
    }
}

// ------------------------------------------------------------------ A4: interpolation

__global__ void k_interp(ResLaunch L, WorkList w, int maxP) {
    if (stage_skipped(L)) return;
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t *V = smem + (size_t)wid * 3 * maxP;
    uint32_t *Wp = V + maxP;
    uint32_t *X = Wp + maxP;     // the integer points x_0 < x_1 < ... actually used
    for (int64_t item = (int64_t)blockIdx.x * nw + wid; item < w.total; item += (int64_t)gridDim.x * nw) {
        int bi = wl_find(w.start, w.n, item);
        int q = w.pairs[bi];
        int i = (int)(item - w.start[bi]);
        const PairPlan &P = L.plan[q];
        const int Pn = P.P;
        const int pt = prime_of(P, L.pmap, i);
        const ModP M = L.mods[pt];
        const uint32_t *g = L.val + P.val_off + (int64_t)i * P.Pe;
        if (P.flag_off < 0) {
            for (int t = lane; t < Pn; t += 32) {
                V[t] = g[t];
                X[t] = (uint32_t)point_of(P.sym, t);
            }
        } else {
            // keep the first Pn points whose flag is clear
            const uint8_t *fl = L.pflags + P.flag_off + (int64_t)i * P.Pe;
            int cnt = 0;
            for (int base = 0; base < P.Pe && cnt < Pn; base += 32) {
                const int j = base + lane;
                const bool good = j < P.Pe && !fl[j];
                const unsigned bal = __ballot_sync(0xffffffffu, good);
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                if (good && pos < Pn) {
                    X[pos] = j;
                    V[pos] = g[j];
                }
                cnt += __popc(bal);
            }
            if (cnt < Pn && lane == 0) atomicExch(L.err, kErrSpareShort);
        }
        for (int t = lane; t < Pn; t += 32) Wp[t] = 0;
        __syncwarp();
        const int C = (Pn + 31) >> 5;
        const int lo0 = lane * C;
        const int hi0 = min(Pn, lo0 + C);
        const uint32_t *inv = L.invk + (int64_t)pt * L.invk_T;
        // divided differences: level k divides by x_j - x_{j-k}, a small positive
        // integer (k on the unit grid), whose inverse comes from the table
        for (int k = 1; k < Pn; ++k) {
            uint32_t prev = (lo0 >= 1 && lo0 - 1 < Pn) ? V[lo0 - 1] : 0u;
            __syncwarp();
            const int lo = max(lo0, k);
            for (int j = hi0 - 1; j >= lo; --j) {
                uint32_t cm1 = (j - 1 >= lo0) ? V[j - 1] : prev;
                const int d = (int)X[j] - (int)X[j - k];   // non-zero, |d| < P
                const uint32_t id = d > 0 ? inv[d] : mp_neg(inv[-d], M.p);
                V[j] = mp_mul(mp_sub(V[j], cm1, M.p), id, M);
            }
            __syncwarp();
        }
        // Newton form -> monomial basis: W = c_{P-1}; W <- W (x - x_k) + c_k
        if (lane == 0) Wp[0] = V[Pn - 1];
        __syncwarp();
        for (int k = Pn - 2; k >= 0; --k) {
            const int deg = Pn - 1 - k;
            const int xk = (int)X[k];
            const uint32_t kt = mp_to(xk >= 0 ? (uint32_t)xk : M.p - (uint32_t)(-xk), M);
            const uint32_t ck = V[k];
            uint32_t prev = (lo0 >= 1 && lo0 - 1 < Pn) ? Wp[lo0 - 1] : 0u;
            __syncwarp();
            const int hi = min(hi0, deg + 1);
            for (int t = hi - 1; t >= lo0; --t) {
                uint32_t below = (t == 0) ? 0u : ((t - 1 >= lo0) ? Wp[t - 1] : prev);
                uint32_t v = mp_sub(below, mp_mul(kt, Wp[t], M), M.p);
                if (t == 0) v = mp_add(v, ck, M.p);
                Wp[t] = v;
            }
            __syncwarp();
        }
        uint32_t *o = L.cf + P.cf_off + (int64_t)i * Pn;
        for (int t = lane; t < Pn; t += 32) o[t] = mp_from(Wp[t], M);
        __syncwarp();
    }
}

// ------------------------------------------------------------------ A4 as a contraction

// Inverse Vandermonde matrix of the points x_j = vinv_point(mode, j), j < n,
// modulo prime i, normal form, row-major: out[(i*n + c)*n + j] = coefficient of
// x^c in the Lagrange basis polynomial L_j(x) = prod_{t != j} (x - x_t) /
// prod_{t != j} (x_j - x_t), times the column scale of the mode.  One block per
// prime: W(x) = prod_t (x - x_t) is built in shared memory, then thread j
// divides W by (x - x_j) (synthetic division) and scales by the inverse of its
// denominator.
__device__ __forceinline__ uint32_t mont_of_int(int v, const ModP &M) {
    return mp_to(v >= 0 ? (uint32_t)v : M.p - (uint32_t)(-v), M);
}

// Point x_j of matrix mode `mode` in Montgomery form (the quartic modes' points
// a^4 exceed 32 bits, so they are formed mod p).
__device__ __forceinline__ uint32_t vinv_point_mont(int mode, int j, const ModP &M) {
    if (mode < VINV_Q0) return mont_of_int(vinv_point(mode, j), M);
    const uint32_t a = mp_to((uint32_t)(mode == VINV_Q0 ? j : j + 1), M), a2 = mp_mul(a, a, M);
    return mp_mul(a2, a2, M);
}

__global__ void k_vinv(const ModP *mods, int n, int mode, uint32_t *out) {
    extern __shared__ uint32_t sh[];
    uint32_t *W = sh;             // n + 1 words, Montgomery form
    const int i = blockIdx.x;
    const ModP M = mods[i];
    for (int t = threadIdx.x; t <= n; t += blockDim.x) W[t] = t == 0 ? M.r1 : 0u;
    __syncthreads();
    for (int j = 0; j < n; ++j) {                 // W <- W (x - x_j), degree j -> j + 1
        const uint32_t jm = vinv_point_mont(mode, j, M);
        uint32_t nv[4];
        int cnt = 0;
        for (int t = threadIdx.x; t <= j + 1 && cnt < 4; t += blockDim.x, ++cnt) {
            uint32_t a = t ? W[t - 1] : 0u, b = t <= j ? W[t] : 0u;
            nv[cnt] = mp_sub(a, mp_mul(jm, b, M), M.p);
        }
        __syncthreads();
        cnt = 0;
        for (int t = threadIdx.x; t <= j + 1 && cnt < 4; t += blockDim.x, ++cnt) W[t] = nv[cnt];
        __syncthreads();
    }
    uint32_t *o = out + (int64_t)i * n * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const uint32_t jm = vinv_point_mont(mode, j, M);
        uint32_t d = M.r1;
        for (int t = 0; t < n; ++t)
            if (t != j) d = mp_mul(d, mp_sub(jm, vinv_point_mont(mode, t, M), M.p), M);
        // column scale 1/2 (EVEN, j >= 1), 1/(2 (j+1)) (ODD), 1/4 (Q0, j >= 1) or
        // 1/(4 (j+1)^t) (Qt) joins the denominator
        if (mode < VINV_Q0) {
            const int den = mode == VINV_EVEN ? (j ? 2 : 1) : mode == VINV_ODD ? 2 * (j + 1) : 1;
            if (den != 1) d = mp_mul(d, mont_of_int(den, M), M);
        } else if (mode > VINV_Q0 || j) {
            uint32_t den = mp_to(4u, M);
            const uint32_t a = mp_to((uint32_t)(j + 1), M);
            for (int t = 0; t < mode - VINV_Q0; ++t) den = mp_mul(den, a, M);
            d = mp_mul(d, den, M);
        }
        const uint32_t id = mp_inv(d, M);
        uint32_t q = W[n];
        o[(int64_t)(n - 1) * n + j] = mp_from(mp_mul(q, id, M), M);
        for (int t = n - 1; t >= 1; --t) {
            q = mp_add(W[t], mp_mul(jm, q, M), M.p);
            o[(int64_t)(t - 1) * n + j] = mp_from(mp_mul(q, id, M), M);
        }
    }
}

// acc += x * y as a 96-bit sum in three words (two multiply-adds with carry and
// one carry add): products are below 2^62, so up to 2^32 of them fit.
__device__ __forceinline__ void mac96(uint32_t &a0, uint32_t &a1, uint32_t &a2, uint32_t x, uint32_t y) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2)
        : "r"(x), "r"(y));
}

constexpr int GT_M = 64, GT_N = 64, GT_K = 32;
static_assert(GT_M == GT_N && GT_M * GT_K % 256 == 0, "one load layout serves both operands");

// coefficients = Vinv_i * operand for one prime i and a group of pairs that
// share the point set.  Tile: 64 coefficient rows x 64 pairs, K in chunks of 32;
// each of the 256 threads owns 4 x 4 outputs.  The operand is the values
// themselves (PLAIN) or, for a complete symmetric point set (value of +i at
// 2i - 1, of -i at 2i), their sums v(i) + v(-i) (EVEN, v(0) for i = 0) or
// differences v(i) - v(-i) (ODD, i = j + 1); sums and differences are formed
// while loading and stay below 2p.  Values are in Montgomery form and Vinv in
// normal form, so the exact sum X = sum Vinv * v~ is congruent to coef * 2^32;
// one reduction per output gives coef.  One block per tile of the flattened
// list of every group's tiles, so all groups share one launch.
__global__ void __launch_bounds__(256, 3) k_interp_gemm(ResLaunch L, const char *planblk, const GemmGroup *groups,
                                                       const GemmTile *tiles) {
    __shared__ uint32_t As[GT_K][GT_M + 1];
    __shared__ __align__(16) uint32_t Bs[GT_K][GT_N + 4];
    if (stage_skipped(L)) return;
    __shared__ uint32_t Cs[GT_N][GT_M + 1];
    __shared__ int64_t colbase[GT_N], cfbase[GT_N];
    const GemmTile T = tiles[blockIdx.x];
    const GemmGroup Gr = groups[T.group];
    const int n = Gr.n, rows = Gr.rows, npairs = Gr.npairs, mode = Gr.mode;
    const int32_t *gpairs = (const int32_t *)(planblk + Gr.pairs_off);
    const uint32_t *vinv = Gr.vinv;
    const int i = T.prime;
    const int c0 = T.c0, q0 = T.q0;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const ModP M = L.mods[i];
    if (threadIdx.x < GT_N) {
        int qi = q0 + threadIdx.x;
        int64_t b = -1;
        if (qi < npairs) {
            const PairPlan &pp = L.plan[gpairs[qi]];
            if (i < pp.k) {
                b = pp.val_off + (int64_t)i * pp.Pe;
                cfbase[threadIdx.x] = pp.cf_off + (int64_t)i * pp.P;
            }
        }
        colbase[threadIdx.x] = b;
    }
    __syncthreads();
    const uint32_t *A = vinv + (int64_t)i * n * n;
    const uint32_t iota = mode >= GEMM_Q0 ? iota_mont(L, i) : 0u;
    uint32_t a0[16], a1[16], a2[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) a0[t] = a1[t] = a2[t] = 0u;
    // the next chunk's operands are loaded into registers while the current
    // chunk is multiplied from shared memory (one chunk of loads in flight)
    constexpr int kLoads = GT_M * GT_K / 256;   // per thread, for A and for B
    uint32_t ra[kLoads], rb[kLoads];
    auto load_chunk = [&](int j0) {
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const int e = threadIdx.x + u * 256;
            const int r = e / GT_K, kk = e % GT_K;
            const int c = c0 + r, j = j0 + kk;
            ra[u] = (c < rows && j < n) ? A[(int64_t)c * n + j] : 0u;
            const int64_t b = colbase[r];
            rb[u] = b >= 0 && j < n ? contraction_operand(L.val + b, mode, j, n, iota, M) : 0u;
        }
    };
    load_chunk(0);
    for (int j0 = 0; j0 < n; j0 += GT_K) {
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const int e = threadIdx.x + u * 256;
            As[e % GT_K][e / GT_K] = ra[u];
            Bs[e % GT_K][e / GT_K] = rb[u];
        }
        __syncthreads();
        if (j0 + GT_K < n) load_chunk(j0 + GT_K);
#pragma unroll 8
        for (int kk = 0; kk < GT_K; ++kk) {
            const uint4 bv = *reinterpret_cast<const uint4 *>(&Bs[kk][tx * 4]);
            const uint32_t av[4] = {As[kk][ty * 4], As[kk][ty * 4 + 1], As[kk][ty * 4 + 2], As[kk][ty * 4 + 3]};
            const uint32_t bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) mac96(a0[r * 4 + cc], a1[r * 4 + cc], a2[r * 4 + cc], av[r], bw[cc]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int t = r * 4 + cc;
            // X * 2^-32 = (a2 2^32 + a1) + a0 2^-32 (mod p); operands below 2p and
            // n <= 8192 terms give (a2:a1) < 2^43 < p 2^32
            uint32_t hi = mp_mul(mp_redc(a1[t], a2[t], M.p, M.pinv), M.r2, M);
            uint32_t lo = mp_redc(a0[t], 0u, M.p, M.pinv);
            Cs[tx * 4 + cc][ty * 4 + r] = mp_add(hi, lo, M.p);
        }
    __syncthreads();
    const int ostride = gemm_ostride(mode), ooff = gemm_ooff(mode);
    for (int e = threadIdx.x; e < GT_N * GT_M; e += 256) {
        int qq = e / GT_M, r = e % GT_M;
        int64_t b = colbase[qq];
        if (b >= 0 && c0 + r < rows) L.cf[cfbase[qq] + (int64_t)(c0 + r) * ostride + ooff] = Cs[qq][r];
    }
}

// ------------------------------------------------------------------ A5: Chinese remaindering

// One thread per output coefficient.  The k residues are read once into this
// thread's column of shared memory (stride BS) and turned into Garner digits
// there; the limbs of the magnitude follow in the same column.  KM = 0 (too
// many primes for shared memory): the digits overwrite the residues in place.
__global__ void k_crt(ResLaunch L, WorkList w, int KM, int LM) {
    if (stage_skipped(L)) return;
    extern __shared__ uint32_t smem[];
    const int BS = blockDim.x;
    uint32_t *limb = smem + (size_t)KM * BS + threadIdx.x;
    for (int64_t item = blockIdx.x * (int64_t)BS + threadIdx.x; item < w.total; item += (int64_t)gridDim.x * BS) {
        int bi = wl_find(w.start, w.n, item);
        int q = w.pairs[bi];
        int c = (int)(item - w.start[bi]);
        const PairPlan &P = L.plan[q];
        const int k = P.k, Pn = P.P;
        const uint32_t *cinv = P.gtab_off < 0 ? L.garner : L.gtab + P.gtab_off;
        const uint32_t *pm = P.gtab_off < 0 ? L.garner + L.garner_K : L.gtab + P.gtab_off + k;
        uint32_t *src = L.cf + P.cf_off + c;
        uint32_t *v = KM ? smem + threadIdx.x : src;
        const int64_t vs = KM ? BS : Pn;
        if (KM)
            for (int i = 0; i < k; ++i) v[i * vs] = src[(int64_t)i * Pn];
        // Garner: digits v_i with X = sum v_i prod_{j<i} p_j, 0 <= v_i < p_i
        for (int i = 1; i < k; ++i) {
            const ModP M = L.mods[prime_of(P, L.pmap, i)];
            const uint32_t *pmi = pm + (int64_t)i * (i - 1) / 2;
            uint32_t t = v[(i - 1) * vs];
            t = min(t, t - M.p);
            for (int j = i - 2; j >= 0; --j) {
                uint32_t vj = v[j * vs];
                vj = min(vj, vj - M.p);
                t = mp_add(mp_mul(t, pmi[j], M), vj, M.p);
            }
            v[i * vs] = mp_mul(mp_sub(v[i * vs], t, M.p), cinv[i], M);
        }
        // symmetric lift: X > (M-1)/2 <=> digits compare above (p_i - 1)/2 from the top
        int cmp = 0;
        for (int i = k - 1; i >= 0 && cmp == 0; --i) {
            uint32_t d = v[i * vs];
            uint32_t h = (L.mods[prime_of(P, L.pmap, i)].p - 1u) >> 1;
            cmp = (d > h) - (d < h);
        }
        const bool neg = cmp > 0;
        // |value| = X or M - X = sum (p_i - 1 - v_i) prod_{j<i} p_j + 1, Horner to 32-bit limbs
        int nl = 0;
        for (int i = k - 1; i >= 0; --i) {
            const uint32_t p = L.mods[prime_of(P, L.pmap, i)].p;
            uint32_t d = v[i * vs];
            if (neg) d = p - 1u - d;
            uint32_t carry = d;
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
        if (nl > P.L) atomicExch(L.err, kErrCrtLimbs);
        uint32_t *o = L.out + P.out_off + (int64_t)c * P.L;
        for (int l = 0; l < P.L; ++l) o[l] = l < nl ? limb[l * BS] : 0u;
        L.sign[P.sign_off + c] = nl == 0 ? 0 : (neg ? -1 : 1);
        if (nl > 0) atomicMax(L.deg + q, c);
    }
}

// Chinese remaindering for pairs on the first kCrtFastK table primes, one
// thread per output coefficient.  Garner digits as dot products:
//   v_i = (r_i - sum_{j<i} v_j prod_{l<j} p_l) (prod_{l<i} p_l)^-1 mod p_i,
// each row summed exactly in 96 bits from the residue r_i R and the table row
// of (-prod_{l<j} p_l) R (one reduction per digit instead of one per term).
// The magnitude X = sum_i v_i prod_{j<i} p_j is built limb by limb from the
// limb table T (limb l = sum_i v_i T[l][i] + carry, exact in 96 bits); a
// negative value has magnitude prod_{i<k} p_i - X, subtracted limb by limb.
// Digits live in shared memory as uint4 groups [i/4][thread], the tables are
// staged in shared memory once per block.
__global__ void k_crt_fast(ResLaunch L, WorkList w, int KD, int LD) {
    if (stage_skipped(L)) return;
    extern __shared__ uint4 smem4[];
    uint32_t *sw = reinterpret_cast<uint32_t *>(smem4);
    const int BS = blockDim.x;
    const int gdw = (crt_gd_off(KD) + 3) & ~3;
    uint32_t *Gd = sw;                                   // gdw words
    uint32_t *T = Gd + gdw;                              // LD rows of kCrtFastRow words
    uint32_t *I0 = T + (size_t)LD * kCrtFastRow;         // LD words (padded to 4)
    uint4 *dig = reinterpret_cast<uint4 *>(I0 + ((LD + 3) & ~3));
    for (int t = threadIdx.x; t < gdw; t += BS) Gd[t] = t < kCrtGdWords ? L.crtfast[t] : 0u;
    for (int t = threadIdx.x; t < LD * kCrtFastRow; t += BS) T[t] = L.crtfast[kCrtGdWords + t];
    for (int t = threadIdx.x; t < LD; t += BS) I0[t] = L.crtfast[kCrtGdWords + kCrtFastL * kCrtFastRow + t];
    __syncthreads();
    uint32_t *dw = reinterpret_cast<uint32_t *>(dig);
    auto dslot = [&](int i) -> uint32_t & { return dw[((size_t)(i >> 2) * BS + threadIdx.x) * 4 + (i & 3)]; };
    // per warp the limbs of its 32 coefficients (pitch LD + 1), written out together
    const int lane = threadIdx.x & 31, opitch = LD + 1;
    uint32_t *ow = reinterpret_cast<uint32_t *>(dig + (size_t)((KD + 3) >> 2) * BS) + (size_t)(threadIdx.x >> 5) * 32 * opitch;
    for (int64_t base = blockIdx.x * (int64_t)BS + threadIdx.x - lane; base < w.total; base += (int64_t)gridDim.x * BS) {
        // a warp's items are consecutive: one search for its first item, and each
        // lane steps over the pair boundaries after it
        int bi = lane == 0 ? wl_find(w.start, w.n, base) : 0;
        bi = __shfl_sync(0xffffffffu, bi, 0);
        const int64_t item = base + lane;
        const bool valid = item < w.total;
        if (valid)
            while (bi + 1 < w.n && item >= w.start[bi + 1]) ++bi;
        const int q = valid ? w.pairs[bi] : -1;
        int top = -1, Lp = 0;    // this coefficient's index if non-zero; its limbs
        int64_t obase = 0;       // where its limbs go
        if (valid) {
            const int c = (int)(item - w.start[bi]);
            const PairPlan &P = L.plan[q];
            const int k = P.k, Pn = P.P, k4 = (k + 3) >> 2;
            const uint32_t *src = L.cf + P.cf_off + c;
            dslot(0) = src[0];
            for (int i = k; i < 4 * k4; ++i) dslot(i) = 0u;   // the last group's unused digits
            for (int i = 1; i < k; ++i) {
                const ModP M = L.mods[i];
                uint32_t a0 = 0u, a1 = src[(int64_t)i * Pn], a2 = 0u;
                const uint4 *row = reinterpret_cast<const uint4 *>(Gd + crt_gd_off(i));
                for (int g = 0; g < ((i + 3) >> 2); ++g) {
                    const uint4 d = dig[(size_t)g * BS + threadIdx.x], e = row[g];
                    mac96(a0, a1, a2, d.x, e.x);
                    mac96(a0, a1, a2, d.y, e.y);
                    mac96(a0, a1, a2, d.z, e.z);
                    mac96(a0, a1, a2, d.w, e.w);
                }
                // (a2 2^32 + a1) + a0 2^-32 = R (r_i - S) 2^-32 = r_i - S (mod p_i)
                const uint32_t hi = mp_mul(mp_redc(a1, a2, M.p, M.pinv), M.r2, M);
                const uint32_t y = mp_add(hi, mp_redc(a0, 0u, M.p, M.pinv), M.p);
                dslot(i) = mp_mul(y, L.garner[i], M);
            }
            // symmetric lift: X > (M-1)/2 <=> digits compare above (p_i - 1)/2 from the top
            int cmp = 0;
            for (int i = k - 1; i >= 0 && cmp == 0; --i) {
                const uint32_t d = dslot(i), h = (L.mods[i].p - 1u) >> 1;
                cmp = (d > h) - (d < h);
            }
            const bool neg = cmp > 0;
            uint32_t *o = ow + lane * opitch;
            uint32_t c0 = 0u, c1 = 0u, borrow = 0u;
            int nl = 0;
            for (int l = 0; l < P.L; ++l) {
                uint32_t a0 = c0, a1 = c1, a2 = 0u;
                const uint32_t *Tl = T + (size_t)l * kCrtFastRow;
                for (int g = (int)(I0[l] >> 2); g < k4; ++g) {
                    const uint4 d = dig[(size_t)g * BS + threadIdx.x];
                    const uint4 e = *reinterpret_cast<const uint4 *>(Tl + 4 * g);
                    mac96(a0, a1, a2, d.x, e.x);
                    mac96(a0, a1, a2, d.y, e.y);
                    mac96(a0, a1, a2, d.z, e.z);
                    mac96(a0, a1, a2, d.w, e.w);
                }
                c0 = a1;
                c1 = a2;
                uint32_t x = a0;
                if (neg) {
                    const uint32_t m = Tl[k];
                    const uint64_t t = (uint64_t)m - x - borrow;
                    x = (uint32_t)t;
                    borrow = (uint32_t)(t >> 63);
                }
                o[l] = x;
                if (x) nl = l + 1;
            }
            L.sign[P.sign_off + c] = nl == 0 ? 0 : (neg ? -1 : 1);
            top = nl > 0 ? c : -1;
            Lp = P.L;
            obase = P.out_off + (int64_t)c * P.L;
        }
        __syncwarp();
        // when the warp's coefficients are consecutive ones of one pair (its valid
        // lanes are a prefix), their limbs are one run of memory: store it
        // coalesced, and raise the pair's degree once
        const int q0 = __shfl_sync(0xffffffffu, q, 0), L0 = __shfl_sync(0xffffffffu, Lp, 0);
        const int64_t ob0 = __shfl_sync(0xffffffffu, obase, 0);
        const bool run = __all_sync(0xffffffffu, !valid || (q == q0 && obase == ob0 + (int64_t)lane * L0));
        if (run) {
            const int nv = __popc(__ballot_sync(0xffffffffu, valid));
            const int tmax = __reduce_max_sync(0xffffffffu, top);
            if (lane == 0 && tmax >= 0) atomicMax(L.deg + q0, tmax);
            int j = lane / L0, l = lane - j * L0;   // word e = j L0 + l of the run
            for (int e = lane; e < nv * L0; e += 32) {
                L.out[ob0 + e] = ow[j * opitch + l];
                for (l += 32; l >= L0; l -= L0) ++j;
            }
        } else if (valid) {
            if (top >= 0) atomicMax(L.deg + q, top);
            for (int l = 0; l < Lp; ++l) L.out[obase + l] = ow[lane * opitch + l];
        }
        __syncwarp();
    }
}

// Chinese remaindering for pairs on the first crtw_K table primes with more than
// kCrtFastK of them, one warp per output coefficient (a one-thread form leaves a few
// hundred coefficients with k^2 serial steps each).  Garner digit i is
//   v_i = (r_i - sum_{j<i} v_j prod_{l<j} p_l) (prod_{l<i} p_l)^-1 mod p_i,
// its dot product split over the lanes (each lane an exact 96-bit sum of its terms with
// the table row (-prod_{l<j} p_l) R mod p_i, lane 0 adding r_i 2^32, reduced to a residue
// mod p_i; the lanes' residues summed by shuffles); the digits stay in shared memory.
// The symmetric lift compares the digits from the top with (p_i - 1) / 2 (a ballot per
// 32 digits); the magnitude X (or prod p_i - X, i.e. the digits p_i - 1 - v_i plus one)
// is sum_i d_i prod_{j<i} p_j: each lane forms the exact 96-bit column sums of its limbs
// from the limb table, and one lane adds them up with their carries.
constexpr int kCrtWarpBlock = 128;
__global__ void __launch_bounds__(kCrtWarpBlock) k_crt_warp(ResLaunch L, WorkList w, int KD, int LD) {
    if (stage_skipped(L)) return;
    extern __shared__ uint32_t smw[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // the primes' constants, staged once per block: p, -p^-1, R^2 mod p, (prod_{j<i} p_j)^-1 R
    uint32_t *cp = smw, *cpinv = cp + KD, *cr2 = cpinv + KD, *cgi = cr2 + KD;
    for (int i = threadIdx.x; i < KD; i += blockDim.x) {
        const ModP M = L.mods[i];
        cp[i] = M.p;
        cpinv[i] = M.pinv;
        cr2[i] = M.r2;
        cgi[i] = L.garner[i];
    }
    __syncthreads();
    uint32_t *dig = smw + 4 * (size_t)KD + (size_t)wib * (KD + 3 * LD);   // KD digits, then LD 96-bit column sums
    uint32_t *col = dig + KD;
    const int KW = L.crtw_K, LW = crt_warp_limbs(KW);
    const uint32_t *T = L.crtw + (size_t)KW * (KW - 1) / 2;
    for (int64_t item = (int64_t)blockIdx.x * nw + wib; item < w.total; item += (int64_t)gridDim.x * nw) {
        const int bi = wl_find(w.start, w.n, item);
        const int q = w.pairs[bi];
        const int c = (int)(item - w.start[bi]);
        const PairPlan &P = L.plan[q];
        const int k = P.k, Pn = P.P, Lp = P.L;
        const uint32_t *src = L.cf + P.cf_off + c;
        __syncwarp();
        for (int i = lane; i < k; i += 32) dig[i] = src[(int64_t)i * Pn];   // residues, then digits in place
        __syncwarp();
        // the first table entry of each row this lane reads (j = lane) is loaded one digit
        // ahead, so that the row's latency overlaps the previous digit's reduction
        uint32_t gnext = lane < 1 ? L.crtw[lane] : 0u;
        for (int i = 1; i < k; ++i) {
            const ModP M{cp[i], cpinv[i], 0u, cr2[i]};
            const uint32_t *Gi = L.crtw + (size_t)i * (i - 1) / 2;
            const uint32_t g0 = gnext;
            if (i + 1 < k) gnext = lane < i + 1 ? Gi[i + lane] : 0u;   // row i + 1 starts i words after row i
            uint32_t a0 = 0u, a1 = lane == 0 ? dig[i] : 0u, a2 = 0u;
            if (lane < i) mac96(a0, a1, a2, dig[lane], g0);
            for (int j = lane + 32; j < i; j += 32) mac96(a0, a1, a2, dig[j], Gi[j]);
            // this lane's (a2 2^64 + a1 2^32 + a0) 2^-32 mod p_i: (a2 2^32 + a1) + a0 2^-32
            uint32_t y = mp_add(mp_mul(mp_redc(a1, a2, M.p, M.pinv), M.r2, M), mp_redc(a0, 0u, M.p, M.pinv), M.p);
            for (int o = 16; o; o >>= 1) y = mp_add(y, __shfl_xor_sync(0xffffffffu, y, o), M.p);
            const uint32_t v = mp_mul(y, cgi[i], M);
            __syncwarp();
            if (lane == 0) dig[i] = v;
            __syncwarp();
        }
        // symmetric lift: X > (M - 1) / 2 <=> the digits compare above (p_i - 1) / 2 from the top
        int cmp = 0;
        for (int base = (k - 1) & ~31; base >= 0; base -= 32) {
            const int i = base + lane;
            int sgn = 0;
            if (i < k) {
                const uint32_t d = dig[i], h = (cp[i] - 1u) >> 1;
                sgn = (d > h) - (d < h);
            }
            const unsigned nz = __ballot_sync(0xffffffffu, sgn != 0);
            if (nz) {
                cmp = __shfl_sync(0xffffffffu, sgn, 31 - __clz(nz));
                break;
            }
        }
        const bool neg = cmp > 0;
        // column sums of limbs l = lane, lane + 32, ...: limb l of prod_{j<i} p_j is zero
        // while prod_{j<i} p_j < 2^(32 l), in particular for 31 i < 32 l (every p_j < 2^31)
        for (int l = lane; l < Lp; l += 32) {
            uint32_t a0 = 0u, a1 = 0u, a2 = 0u;
#pragma unroll 4
            for (int i = (32 * l) / 31; i < k; ++i) {
                uint32_t d = dig[i];
                if (neg) d = cp[i] - 1u - d;
                mac96(a0, a1, a2, d, T[(size_t)i * LW + l]);
            }
            col[3 * l] = a0;
            col[3 * l + 1] = a1;
            col[3 * l + 2] = a2;
        }
        __syncwarp();
        int nl = 0;
        bool over = false;
        if (lane == 0) {
            // limb l of X (plus one for a negative value) = column l plus the carry; col[l]
            // takes the limb once column l / 3 (<= l) has been read
            unsigned __int128 acc = neg ? 1u : 0u;
            for (int l = 0; l < Lp; ++l) {
                acc += (unsigned __int128)col[3 * l] | ((unsigned __int128)col[3 * l + 1] << 32) |
                       ((unsigned __int128)col[3 * l + 2] << 64);
                const uint32_t limb = (uint32_t)acc;
                acc >>= 32;
                col[l] = limb;
                if (limb) nl = l + 1;
            }
            over = acc != 0;
        }
        __syncwarp();
        nl = __shfl_sync(0xffffffffu, nl, 0);
        over = __shfl_sync(0xffffffffu, over, 0);
        uint32_t *o = L.out + P.out_off + (int64_t)c * Lp;
        for (int l = lane; l < Lp; l += 32) o[l] = col[l];
        if (lane == 0) {
            if (over) atomicExch(L.err, kErrCrtLimbs);
            L.sign[P.sign_off + c] = nl == 0 ? 0 : (neg ? -1 : 1);
            if (nl > 0) atomicMax(L.deg + q, c);
        }
    }
}

// ------------------------------------------------------------------ A6: unlucky primes

// Flags prime c of pair q when the leading row of f or of g vanishes identically
// modulo it (then every evaluation point of that prime is unlucky).  For disc,
// lc(df/dy) = m lc(f) and the table primes exceed m, so f's row decides.
__global__ void k_unlucky_primes(ResLaunch L, int kc, uint8_t *out) {
    const int64_t total = (int64_t)L.npairs * kc;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(it / kc), c = (int)(it % kc);
        const PairBound &B = L.bounds[q];
        const PairDesc &D = L.desc[q];
        uint8_t bad = 0;
        if (B.m >= 0 && B.n >= 0) {
            const ModP M = L.mods[c];
            for (int w = 0; w < 2 && !bad; ++w) {
                if (w == 1 && D.disc) break;
                const PolyDesc &Pd = w ? D.g : D.f;
                const int row = w ? B.n : B.m;
                bool allzero = true;
                for (int col = 0; col <= Pd.cols && allzero; ++col)
                    allzero = mp_from_words(coef_ptr(L.coef, Pd, row, col), Pd.words, M) == 0u;
                bad = allzero;
            }
        }
        out[it] = bad;
    }
}

// Garner constants of a pair whose primes are not a prefix of the table
// (same layout as the prefix table: k inverses, then the triangle).
__global__ void k_pair_garner(ResLaunch L, const int32_t *pairs, int n, int kmax, uint32_t *gtab) {
    if (stage_skipped(L)) return;
    const int64_t total = (int64_t)n * kmax;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
        const PairPlan &P = L.plan[pairs[it / kmax]];
        const int i = (int)(it % kmax), k = P.k;
        if (i >= k) continue;
        const ModP M = L.mods[prime_of(P, L.pmap, i)];
        uint32_t *tab = gtab + P.gtab_off;
        uint32_t *pm = tab + k + (int64_t)i * (i - 1) / 2;
        uint32_t prod = M.r1;
        for (int j = 0; j < i; ++j) {
            uint32_t pj = L.mods[prime_of(P, L.pmap, j)].p;
            pj = pj >= M.p ? pj - M.p : pj;
            uint32_t pjm = mp_to(pj, M);
            pm[j] = pjm;
            prod = mp_mul(prod, pjm, M);
        }
        tab[i] = mp_inv(prod, M);
    }
}

// ------------------------------------------------------------------ launchers

// The dynamic shared-memory ceiling of every kernel is raised once, to the same
// value, when a context is created: changing it per launch would race between
// host threads that launch concurrently (serving workers).
cudaError_t configure_res_kernels() {
    cudaError_t e = configure_evalres_kernel();
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_interp, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_crt, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_crt_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_crt_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_vinv, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    return e;
}

cudaError_t launch_reduce(const ResLaunch &L, const WorkList &w, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    int block = 256;
    int grid = persistent_grid(k_reduce, block, 0, (w.total + block - 1) / block);
    k_reduce<<<grid, block, 0, s>>>(L, w);
    return cudaGetLastError();
}

cudaError_t launch_interp(const ResLaunch &L, const WorkList &w, int maxP, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    size_t per_warp = (size_t)3 * maxP * sizeof(uint32_t);
    int nw = (int)((48 * 1024) / per_warp);
    if (nw > 8) nw = 8;
    if (nw < 1) nw = 1;
    size_t smem = per_warp * nw;
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    int grid = persistent_grid(k_interp, nw * 32, smem, (w.total + nw - 1) / nw);
    k_interp<<<grid, nw * 32, smem, s>>>(L, w, maxP);
    return cudaGetLastError();
}

cudaError_t launch_vinv(const ModP *mods, int n, int K, int mode, uint32_t *out, cudaStream_t s) {
    if (n < 1) return cudaErrorInvalidValue;
    size_t smem = (size_t)(n + 1) * sizeof(uint32_t);
    int block = n + 2 <= 1024 ? ((n + 2 + 31) / 32) * 32 : 1024;
    // each thread updates at most 4 coefficients of W per step
    if (smem > kMaxDynSmem || n + 1 > 4 * block) return cudaErrorInvalidValue;
    k_vinv<<<K, block, smem, s>>>(mods, n, mode, out);
    return cudaGetLastError();
}

cudaError_t launch_interp_gemm(const ResLaunch &L, const char *planblk, const GemmGroup *groups,
                               const GemmTile *tiles, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    k_interp_gemm<<<ntiles, 256, 0, s>>>(L, planblk, groups, tiles);
    return cudaGetLastError();
}

cudaError_t launch_crt_fast(const ResLaunch &L, const WorkList &w, int maxK, int maxL, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    if (maxK > kCrtFastK || maxL > kCrtFastL) return cudaErrorInvalidValue;
    const int block = 128, k4 = (maxK + 3) / 4;
    const size_t tab = (size_t)((crt_gd_off(maxK) + 3) & ~3) + (size_t)maxL * kCrtFastRow + ((maxL + 3) & ~3);
    // tables, digits (k4 per thread) and the staged output limbs (maxL + 1 per thread)
    const size_t smem = tab * 4 + (size_t)k4 * block * 16 + (size_t)block * (maxL + 1) * 4;
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    int grid = persistent_grid(k_crt_fast, block, smem, (w.total + block - 1) / block);
    k_crt_fast<<<grid, block, smem, s>>>(L, w, maxK, maxL);
    return cudaGetLastError();
}

cudaError_t launch_unlucky_primes(const ResLaunch &L, int kc, uint8_t *out, cudaStream_t s) {
    int64_t total = (int64_t)L.npairs * kc;
    if (total <= 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_unlucky_primes<<<grid, 256, 0, s>>>(L, kc, out);
    return cudaGetLastError();
}

cudaError_t launch_pair_garner(const ResLaunch &L, const int32_t *pairs, int n, int kmax, uint32_t *gtab,
                               cudaStream_t s) {
    int64_t total = (int64_t)n * kmax;
    if (total <= 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_pair_garner<<<grid, 256, 0, s>>>(L, pairs, n, kmax, gtab);
    return cudaGetLastError();
}

cudaError_t launch_crt_warp(const ResLaunch &L, const WorkList &w, int maxK, int maxL, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    if (maxK > L.crtw_K || !L.crtw) return cudaErrorInvalidValue;
    const size_t smem = (4 * (size_t)maxK + (size_t)(kCrtWarpBlock / 32) * (maxK + 3 * maxL)) * sizeof(uint32_t);
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    const int64_t blocks = (w.total + kCrtWarpBlock / 32 - 1) / (kCrtWarpBlock / 32);
    const int grid = persistent_grid(k_crt_warp, kCrtWarpBlock, smem, blocks);
    k_crt_warp<<<grid, kCrtWarpBlock, smem, s>>>(L, w, maxK, maxL);
    return cudaGetLastError();
}

cudaError_t launch_crt(const ResLaunch &L, const WorkList &w, int maxK, int maxL, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    int block = 128;
    while (block > 32 && (size_t)(maxK + maxL) * block * 4 > 160 * 1024) block >>= 1;
    if ((size_t)(maxK + maxL) * block * 4 > 160 * 1024) maxK = 0;   // digits stay in global memory
    // results of more than 1280 limbs (about 1320 primes): fewer threads per block,
    // below a warp if need be (every thread works alone, no warp-wide operation)
    while (block > 1 && (size_t)maxL * block * 4 > 160 * 1024) block >>= 1;
    size_t smem = (size_t)(maxK + maxL) * block * sizeof(uint32_t);
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    int grid = persistent_grid(k_crt, block, smem, (w.total + block - 1) / block);
    k_crt<<<grid, block, smem, s>>>(L, w, maxK, maxL);
    return cudaGetLastError();
}

}  // namespace gbr
