// Internal structures shared by the host driver and the kernels of libgbres.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/gbres.h"
#include "gbr_modarith.cuh"

namespace gbr {

// Codes the resultant kernels leave in the context's device error word (the
// call then returns GBR_EDEVICE with the matching message).
constexpr int kErrCrtLimbs = 2;       // a lifted coefficient needed more limbs than planned
constexpr int kErrSpareShort = 5;     // drop mode ran out of spare points
constexpr int kErrTensorStall = 6;    // a tensor-core wait gave up (interpolation skipped its results)
constexpr int kErrNttDegree = 8;      // an inverse transform left a coefficient above the degree bound

// ------------------------------------------------------------------ prime table (host)
int num_primes();
const ModP *host_mods();              // ModP for every table prime, p_0 > p_1 > ...
size_t prime_table_bytes();             // device prime table: ModP[num_primes()], uint2 (R^3, R^4)[num_primes()],
// the device prime table's bytes, built on the host (layout of prime_table_bytes)
void build_prime_table(std::vector<char> &buf);
cudaError_t upload_prime_table(ModP *d);  // then the CRT tables of the first kCrtFastK primes
const uint2 *prime_r34(const ModP *d);
const uint32_t *prime_crt_tables(const ModP *d);
const uint32_t *prime_roots(const ModP *d);

// Roots of unity.  Every table prime is 1 mod 2^kRootLog, so it has a root of
// unity w of order 2^kRootLog (w^(2^(kRootLog - 1)) = -1).  The device prime
// table holds per prime kRootTabWords words: T1[j] = w^j R mod p and
// T2[j] = w^(128 j) R mod p for j < 128 (Montgomery forms), so that
// w^e R = mp_mul(T1[e mod 128], T2[e / 128]) for every e < 2^kRootLog.
constexpr int kRootLog = 14;
constexpr int kRootOrder = 1 << kRootLog;
constexpr int kRootTabWords = 256;
GBR_HD uint32_t root_pow(const uint32_t *tab, int e, const ModP &M) {
    return mp_mul(tab[e & 127], tab[128 + (e >> 7)], M);
}

// Chinese remaindering tables for pairs on the first kCrtFastK table primes:
//   Garner rows: row i (at crt_gd_off(i), padded with zeros to a multiple of 4)
//     holds (-prod_{l<j} p_l mod p_i) R mod p_i for j < i, so that
//     r_i R + sum_j v_j row_i[j] = R (r_i - sum_{j<i} v_j prod_{l<j} p_l) (mod p_i);
//   limb table T[l][i] (rows of kCrtFastRow words): limb l of prod_{j<i} p_j, i <= kCrtFastK;
//   I0[l]: the first i (a multiple of 4) with T[l][i] != 0.
constexpr int kCrtFastK = 64, kCrtFastRow = 68, kCrtFastL = 62;
GBR_HD int crt_gd_off(int i) {
    if (i <= 0) return 0;
    const int q = (i - 1) / 4, r = (i - 1) % 4;
    return 8 * q * (q + 1) + 4 * r * (q + 1);
}
constexpr int kCrtGdWords = 8 * 15 * 16 + 4 * 3 * 16;   // crt_gd_off(kCrtFastK)
constexpr int kCrtTabWords = kCrtGdWords + kCrtFastL * kCrtFastRow + kCrtFastL;
double log2_prime_prefix(int k);      // sum_{i<k} log2 p_i
int primes_for_bits(double bits);     // smallest k with sum_{i<k} log2 p_i > bits

// Garner constants for the prefix prime list p_0..p_{k-1}: for prime i,
// cinv[i] = (p_0 ... p_{i-1})^-1 mod p_i and pm[i*(i-1)/2 + j] = p_j mod p_i (j < i),
// both in Montgomery form modulo p_i.  Layout: cinv[0..K) then pm.
void garner_prefix_table(int K, uint32_t *out);   // out has K + K*(K-1)/2 words
// Tables of the warp-per-coefficient Chinese remaindering for pairs on the first K
// (kCrtFastK < K <= kCrtWarpK) table primes: Garner rows, row i (at i(i-1)/2) holding
// (-prod_{l<j} p_l mod p_i) R mod p_i for j < i, then the limb table, row i (i < K,
// crt_warp_limbs(K) words each) holding the 32-bit limbs of prod_{j<i} p_j.
constexpr int kCrtWarpK = 512;
// every prime is below 2^31, so prod_{j<i} p_j with i <= K fits (31 K + 31) / 32 limbs
GBR_HD int crt_warp_limbs(int K) { return (31 * K + 31) / 32; }
size_t crt_warp_words(int K);
void crt_warp_table(int K, uint32_t *out);

// Inverses 1/t mod p_i for t = 1..T-1 in Montgomery form, t = 0 slot unused:
// out[i*T + t].
void inverse_table(int K, int T, uint32_t *out);

// ------------------------------------------------------------------ resident batch
// One input polynomial in the eliminated-variable view: row r is the coefficient
// of (eliminated variable)^r, column c the power of the other variable.
struct PolyDesc {
    int64_t off;        // first 64-bit word of the polynomial in the coefficient buffer
    int32_t rows;       // row extent (number of rows - 1)
    int32_t cols;       // column extent
    int32_t rstride;    // coefficient stride between rows
    int32_t cstride;    // coefficient stride between columns
    int32_t words;      // 64-bit words per coefficient
    int32_t rowdeg_off; // where the bounds kernel writes this polynomial's row degrees
};

struct PairDesc {
    PolyDesc f, g;      // for disc, g is unused: g_j = (j+1) f_{j+1}
    int32_t disc;
    int32_t pad;
};

// Written by the bounds kernel (one per pair), read back by the host planner.
struct PairBound {
    int32_t m, n;       // actual degrees in the eliminated variable (-1: zero polynomial)
    int32_t dxf, dxg;   // actual degrees in the other variable
    int32_t tdf, tdg;   // total degrees
    int32_t tf, tg;     // Horner terms: sum over rows <= degree of (row degree + 1)
    int32_t lcdf, lcdg; // degrees (in the other variable) of the leading coefficients
    int32_t pad;
    double log2B;       // upper bound on log2 of the Hadamard bound
};

// Per-pair plan, written by the host, read by every stage kernel.
struct PairPlan {
    int32_t m, n, dxf, dxg;
    int32_t P;          // interpolation points = degree bound + 1
    int32_t Pe;         // evaluated points: P, or P + spares when unlucky points are dropped
    int32_t k;          // primes
    int32_t L;          // 32-bit limbs per output coefficient
    int32_t S;          // residue words per prime: (dxf+1) rows4(m) + (dxg+1) rows4(n)
    int32_t pmap_off;   // -1: primes are table entries 0..k-1; else their table indices at pmap[pmap_off..]
    int32_t sym;        // point set (PTS_*): PTS_SYM points are point_of(j) (0, 1, -1, 2, -2, ...),
                        // PTS_ROOTS points are u^j (u a primitive Pe-th root of unity); both are
                        // evaluated in +-a lane pairs
    int32_t tiles;      // PTS_SYM, PTS_ROOTS: warp tiles of 16 lane pairs per prime; PTS_QUAD:
                        // warps over all primes (quad_warps)
    int64_t res_off;    // residues [prime][S]                       (u32 words)
    int64_t val_off;    // values [prime][Pe]                        (u32 words)
    int64_t cf_off;     // coefficients mod p [prime][P]             (u32 words)
    int64_t flag_off;   // -1, or unlucky-point flags [prime][Pe]    (bytes)
    int64_t gtab_off;   // -1: prefix Garner table; else this pair's table (k + k(k-1)/2 words)
    int64_t out_off;    // output magnitudes [coef][L]               (u32 words)
    int64_t sign_off;   // output signs [coef]                       (bytes)
    int32_t rowdeg_f, rowdeg_g;   // offsets of row degree arrays
    int32_t disc, flags;          // flags bit0: zero result, no device work
};

enum : int32_t { PLAN_ZERO = 1 };

// Point sets: the unit grid 0..Pe-1 (drop mode), the symmetric integers
// 0, +-1, +-2, ..., the Pe-th roots of unity u^j with Pe a power of two
// (interpolated by an inverse transform), or the quartic set 0, +-a, +-i a
// (a = 1..h, i^2 = -1 mod p), whose values at i^k a give the four quarter parts
// R_t of R(x) = sum_t x^t R_t(x^4) by a 4-point transform.
enum : int32_t { PTS_GRID = 0, PTS_SYM = 1, PTS_ROOTS = 2, PTS_QUAD = 3 };

// Quartic set: value index 4 (a - 1) + k is x = i^k a (k = 0: a, 1: i a, 2: -a,
// 3: -i a; a = 1..h), index 4 h is x = 0, and 4 h + 1 .. 4 h + 3 are pads (they
// receive copies of the value at 0), so that a point quadruple is 16-byte aligned
// (the planner aligns a quartic pair's values to 4 words) and the interpolation
// loads it at once.  The evaluation kernels take the set by quadruples: quadruple
// Q = i (h + 1) + a of a pair holds the points i^k a of prime i (a = 0: the point 0
// and the pads), the pair's quadruples over all its primes are laid out flat, eight
// to a warp (quad_warps warps per pair; a warp may span two primes), and the four
// points of one quadruple stay in one warp.
GBR_HD int quad_h(int P) { return (P - 1 + 3) / 4; }          // a = 1..h covers P - 1 points
GBR_HD int quad_pe(int P) { return 4 * quad_h(P) + 4; }
GBR_HD int quad_pairs(int P) { return 2 * quad_h(P) + 1; }    // +-x lane pairs
GBR_HD int quad_warps(int P, int k) { return (int)(((int64_t)k * (quad_h(P) + 1) + 7) / 8); }
// Lane `lane` of warp w of a pair's quartic work: its quadruple's prime i (clamped
// to k - 1 past the last one), base a, and whether the quadruple exists.
struct QuadLane {
    int i, a, h;
    bool live;
};
GBR_HD QuadLane quad_lane(int P, int k, int64_t w, int qi) {
    const int h = quad_h(P), hq = h + 1;
    const int64_t Q = w * 8 + qi;
    QuadLane r;
    r.h = h;
    r.live = Q < (int64_t)k * hq;
    r.i = r.live ? (int)(Q / hq) : k - 1;
    r.a = r.live ? (int)(Q - (int64_t)r.i * hq) : 0;
    return r;
}
// value index of the point i^kk a of a quadruple (a = 0: the point 0 and the pads;
// -1: none)
GBR_HD int quad_index(const QuadLane &q, int kk) {
    return !q.live ? -1 : q.a == 0 ? 4 * q.h + kk : 4 * (q.a - 1) + kk;
}
// coefficients of the quarter part R_t of a resultant with P coefficients (degree P - 1)
GBR_HD int quad_rows(int P, int t) { return P - 1 >= t ? (P - 1 - t) / 4 + 1 : 0; }

// Residue rows of a polynomial of degree m in the eliminated variable, padded to
// a multiple of 4 (the evaluation reads four rows per 16-byte load).
GBR_HD int32_t rows4(int32_t m) { return (m + 1 + 3) & ~3; }

// Upper bound on log2 |coefficient| of res_y(f, g), from Hadamard's inequality on
// the unit circle |x| = 1 (a coefficient of R is at most max |R(x)| there, and
// |f_i(x)| <= ||f_i||_1).  lf[i] = log2 ||f_i||_1 (i = 0..m, -inf for zero
// rows), lg likewise.  For any lambda > 0, res(f(x, lambda y), g(x, lambda y)) =
// lambda^(mn) res(f, g), so the Hadamard bound of the scaled Sylvester matrix
// (entries lambda^i f_i) minus mn log2 lambda is a bound too; both the product
// of row norms and the product of column norms are used, and the smaller is
// returned.  l2lam = log2 lambda.
GBR_HD double scaled_hadamard_log2(const double *lf, int m, const double *lg, int n, double l2lam, double *ef,
                                   double *eg) {
    if (m <= 0 && n <= 0) return 0.0;
    // scaled log2 norms, their maximum, and 2^(2 (F_i - M)) clamped below at
    // 2^-1000 (enlarging a term only enlarges the bound; no sum underflows)
    double M = -INFINITY;
    for (int i = 0; i <= m; ++i)
        if (lf[i] != -INFINITY && lf[i] + i * l2lam > M) M = lf[i] + i * l2lam;
    for (int j = 0; j <= n; ++j)
        if (lg[j] != -INFINITY && lg[j] + j * l2lam > M) M = lg[j] + j * l2lam;
    double sf = 0.0, sg = 0.0;
    for (int i = 0; i <= m; ++i) {
        double t = lf[i] == -INFINITY ? 0.0 : exp2(fmax(2.0 * (lf[i] + i * l2lam - M), -1000.0));
        ef[i] = t;
        sf += t;
    }
    for (int j = 0; j <= n; ++j) {
        double t = lg[j] == -INFINITY ? 0.0 : exp2(fmax(2.0 * (lg[j] + j * l2lam - M), -1000.0));
        eg[j] = t;
        sg += t;
    }
    double row = 0.0;
    if (n > 0) row += 0.5 * n * (2.0 * M + log2(sf));
    if (m > 0) row += 0.5 * m * (2.0 * M + log2(sg));
    double col = 0.0;
    for (int c = 0; c < m + n; ++c) {
        double sc = 0.0;
        // f rows r = 0..n-1 hold f_{m-(c-r)} in column c when 0 <= c - r <= m
        int r0 = c - m > 0 ? c - m : 0, r1 = c < n - 1 ? c : n - 1;
        for (int r = r0; r <= r1; ++r) sc += ef[m - (c - r)];
        // g rows r = 0..m-1 hold g_{n-(c-r)} when 0 <= c - r <= n
        r0 = c - n > 0 ? c - n : 0;
        r1 = c < m - 1 ? c : m - 1;
        for (int r = r0; r <= r1; ++r) sc += eg[n - (c - r)];
        col += sc > 0.0 ? 0.5 * (2.0 * M + log2(sc)) : -INFINITY;
    }
    double b = row < col ? row : col;
    // sums of k non-negative doubles carry a relative error below k 2^-53; the
    // planner adds two bits and a relative margin on top of this value
    return b - (double)m * n * l2lam;
}

// log2 lambda values the planner tries (the bound is valid for each; the
// smallest is used)
constexpr int kBoundLambdas = 13;
// (0, 0.25, 0.5, 0.75, 1, 1.5, 2, 3, 4, 5, 6, -0.5, -1), computed rather than
// indexed so that no table lands in a kernel's local memory
GBR_HD double bound_lambda(int l) {
    return l < 5 ? 0.25 * l : l < 7 ? 1.0 + 0.5 * (l - 4) : l < 11 ? (double)(l - 4) : -0.5 * (l - 10);
}

// the same values in single precision (all exact), for device code
GBR_HD float bound_lambda_f(int l) {
    return l < 5 ? 0.25f * l : l < 7 ? 1.0f + 0.5f * (l - 4) : l < 11 ? (float)(l - 4) : -0.5f * (l - 10);
}

GBR_HD double best_scaled_bound(const double *lf, int m, const double *lg, int n, double *ef, double *eg) {
    if (m <= 0 && n <= 0) return 0.0;
    double best = INFINITY;
    for (int l = 0; l < kBoundLambdas; ++l) {
        double b = scaled_hadamard_log2(lf, m, lg, n, bound_lambda(l), ef, eg);
        if (b < best) best = b;
    }
    return best;
}

// Host-side bound arithmetic shared by gbr_resultant_info and the planner.
GBR_HD int32_t degree_bound(const PairBound &b) {
    if (b.m < 0 || b.n < 0) return 0;
    int64_t d1 = (int64_t)b.n * b.dxf + (int64_t)b.m * b.dxg;
    int64_t d2 = (int64_t)b.tdf * b.tdg;
    int64_t d = d1 < d2 ? d1 : d2;
    return (int32_t)(d < 0 ? 0 : d);
}

// Size of a root-of-unity point set for P coefficients: the next power of two,
// at least 64 (two warp tiles of lane pairs).
GBR_HD int root_points(int P) {
    int N = 64;
    while (N < P) N <<= 1;
    return N;
}

// Shared point counts of a batch.  counts: the batch's distinct point counts in
// ascending order with their numbers of pairs.  Returns the count each one is raised to:
// runs of consecutive counts take the run's largest, a run growing while it holds fewer
// than `tile` pairs and the next count stays within 1/16 (at least 4 points) above the
// run's smallest and, from 512 points on (where roots of unity can pay), needs the
// same root-of-unity set (root_points), so that a pair evaluated at roots of unity never
// doubles its points.  (A contraction group of a few
// pairs costs about as much as a full tile; a degree bound may always be raised.)
inline std::vector<int32_t> share_point_counts(const std::vector<std::pair<int32_t, int>> &counts, int tile) {
    std::vector<int32_t> to(counts.size());
    size_t start = 0;
    int64_t acc = 0;
    for (size_t i = 0; i < counts.size(); ++i) {
        acc += counts[i].second;
        const int32_t lo = counts[start].first;
        const bool more = i + 1 < counts.size() && acc < tile &&
                          counts[i + 1].first <= lo + (lo / 16 > 4 ? lo / 16 : 4) &&
                          (lo < 512 || root_points(counts[i + 1].first) == root_points(lo));
        if (more) continue;
        for (size_t j = start; j <= i; ++j) to[j] = counts[i].first;
        start = i + 1;
        acc = 0;
    }
    return to;
}

// Whether root-of-unity points pay for a pair with P coefficients (N points),
// y-degrees m, n and t_f, t_g stored coefficients, `share` pairs of the batch
// having the same P, by an estimate in modular products per (pair, prime): the
// N - P extra points cost their evaluation ((t_f + t_g) / 2 Horner steps) and
// elimination (about 1.5 m n products plus the inverse), the inverse transform
// about 5 N log2 N (it is memory and barrier bound); the integer points'
// inverse-Vandermonde contraction costs P^2 / 2 multiply-adds (even and odd
// halves; P^2 / 4 for the four quarter parts of a quartic set) at about half a
// product each on the tensor cores (matrices up to 256 points, tiles of 128 pairs)
// and 0.85 on the integer pipes (tiles of 64 pairs), inflated by the unused part of
// its last tile;
// above 4097 points the integer points fall back to Newton interpolation, which
// one warp per (pair, prime) runs far slower.  (Constants fitted to the
// measured crossover of this GPU.)
GBR_HD bool roots_pay(int P, int N, int tf, int tg, int m, int n, int share, bool tc, bool gemm, bool quad) {
    const double per_point = 0.5 * (tf + tg) + 1.5 * m * n + 5.0 * (m > n ? m : n) + 50.0;
    int lg = 0;
    while ((1 << lg) < N) ++lg;
    const double roots = per_point * (N - P) + 5.0 * N * lg;
    if (!gemm || P > 4097) return true;
    const int s = share < 1 ? 1 : share;
    const bool on_tc = (quad ? P <= 1021 : P <= 511) && tc;
    const int tile = on_tc ? 128 : 64;
    const double tile_waste = (double)((s + tile - 1) / tile * tile) / s;
    const double per_mac = (on_tc ? 0.5 : 0.85) * tile_waste;
    return roots < per_mac * (quad ? 0.25 : 0.5) * (double)P * P;
}

// ------------------------------------------------------------------ kernel launchers
struct ResLaunch {
    // device pointers
    const uint64_t *coef;
    const PairDesc *desc;
    PairBound *bounds;
    int32_t *rowdeg;
    const PairPlan *plan;
    const ModP *mods;
    const uint2 *r34;            // per prime (R^3 mod p, R^4 mod p), R = 2^32
    const uint32_t *roots;       // per prime kRootTabWords words of root-of-unity powers
    const uint32_t *crtfast;     // CRT tables of the first kCrtFastK primes (Garner rows, T, I0)
    const uint32_t *garner;      // prefix Garner table (K + K(K-1)/2 words)
    int32_t garner_K;
    const uint32_t *crtw;        // warp Chinese remaindering tables of the first crtw_K primes
    int32_t crtw_K;
    const uint32_t *invk;        // [prime][invk_T] inverses of 1..T-1
    int32_t invk_T;
    uint32_t *res;               // residues
    uint32_t *val;               // values R(a) mod p at the points (Montgomery form; numerators until
                                 // k_batch_inv divides them by den)
    uint32_t *den;               // denominators of the values (Montgomery form, non-zero), same layout
    uint32_t *cf;                // coefficients of R mod p (normal form), same offsets as val
    uint32_t *out;               // output magnitudes
    int8_t *sign;                // output signs
    int32_t *deg;                // per pair output degree
    int32_t *err;                // device error word (0 = ok)
    const int32_t *pmap;         // per-pair prime maps (drop mode)
    uint8_t *pflags;             // unlucky-point flags (drop mode)
    const uint32_t *gtab;        // per-pair Garner tables (drop mode)
    unsigned long long *dropped; // count of flagged points
    const int32_t *skip;         // null, or a device flag: non-zero makes every stage kernel return at once
                                 // (a replayed step whose plan no longer matches its bounds)
    int32_t npairs;
    int32_t drop_unlucky;
};

// Evaluation point j: the unit grid j, or the symmetric order 0, 1, -1, 2, -2, ...
__host__ __device__ __forceinline__ int point_of(int sym, int j) {
    return !sym ? j : ((j & 1) ? (j + 1) >> 1 : -(j >> 1));
}

__host__ __device__ __forceinline__ int prime_of(const PairPlan &P, const int32_t *pmap, int i) {
    return P.pmap_off < 0 ? i : pmap[P.pmap_off + i];
}

// Work lists (device arrays, built by the host planner).
struct WorkList {
    const int32_t *pairs;     // pair ids
    const int64_t *start;     // start[i] = first item of pairs[i]; start[n] = total
    int32_t n;
    int64_t total;
};

// pairs sharing a point count needed before interpolation uses the contraction
// (its inverse Vandermonde matrix is cached per point count; Newton is the
// fallback when the matrix cannot be cached)
constexpr int kGemmMinPairs = 1;

// dynamic shared memory ceiling set once for every kernel (bytes)
constexpr int kMaxDynSmem = 200 * 1024;
cudaError_t configure_res_kernels();
cudaError_t configure_evalres_kernel();
cudaError_t configure_gcd_kernels();
cudaError_t configure_sqf_kernels();

cudaError_t launch_bounds(const ResLaunch &L, cudaStream_t s);
// *flag = 1 when the fresh bounds of some pair no longer fit its plan (degrees, points or
// primes); l2pref[k] = sum_{i<k} log2 p_i on the device
cudaError_t launch_plan_check(const PairBound *bounds, const PairPlan *plan, int n, const double *l2pref,
                              int extra, int32_t *flag, cudaStream_t s);
// true when a replayed step must not run its stages
__device__ __forceinline__ bool stage_skipped(const ResLaunch &L) { return L.skip && *(volatile const int32_t *)L.skip; }
cudaError_t launch_reduce(const ResLaunch &L, const WorkList &w, cudaStream_t s);
cudaError_t launch_evalres(const ResLaunch &L, const WorkList &w, int slots_f, int slots_g, int block,
                           cudaStream_t s);
// register form for symmetric pairs of shape (N, N), (N, N-1), (N-1, N) with
// kRegMinN <= N <= kRegMaxN; warps it cannot finish are listed in `redo`
// (capacity total / 32, count in *redo_n, zeroed before) and solved by a
// second launch on shared memory
constexpr int kRegMinN = 2, kRegMaxN = 32;
GBR_HD int reg_shape(int m, int n) {
    const int N = m > n ? m : n;
    if (N < kRegMinN || N > kRegMaxN || m < N - 1 || n < N - 1) return 0;
    return N;
}
cudaError_t launch_evalres_reg(const ResLaunch &L, const WorkList &w, int N, int block, unsigned long long *redo_n,
                               int64_t *redo, cudaStream_t s);
cudaError_t launch_interp(const ResLaunch &L, const WorkList &w, int maxP, cudaStream_t s);
// values = numerators / denominators, one warp per (pair, prime, segment of
// kInvSegment values) of the work list (Montgomery's batch inversion)
constexpr int kInvSegment = 512;
cudaError_t launch_batch_inv(const ResLaunch &L, const WorkList &w, cudaStream_t s);
// inverse transform for PTS_ROOTS pairs (one item per (pair, prime)); maxN = largest Pe
cudaError_t launch_interp_ntt(const ResLaunch &L, const WorkList &w, int maxN, cudaStream_t s);
cudaError_t configure_interp_ntt_kernel();
cudaError_t launch_crt(const ResLaunch &L, const WorkList &w, int maxK, int maxL, cudaStream_t s);
// pairs on the prime-table prefix with k <= kCrtFastK
cudaError_t launch_crt_fast(const ResLaunch &L, const WorkList &w, int maxK, int maxL, cudaStream_t s);
cudaError_t launch_crt_warp(const ResLaunch &L, const WorkList &w, int maxK, int maxL, cudaStream_t s);
cudaError_t launch_vinv(const ModP *mods, int n, int K, int mode, uint32_t *out, cudaStream_t s);
cudaError_t launch_unlucky_primes(const ResLaunch &L, int kc, uint8_t *out, cudaStream_t s);
cudaError_t launch_pair_garner(const ResLaunch &L, const int32_t *pairs, int n, int kmax, uint32_t *gtab,
                               cudaStream_t s);
// Interpolation as a contraction: pairs sharing a point count form a group;
// the launch covers tiles of 64 coefficients x 64 pairs x one prime.
// Point sets of the inverse Vandermonde matrices (k_vinv):
//   VINV_GRID  x_j = j                       (values at the unit grid)
//   VINV_SYM   x_j = point_of(1, j)          (values at 0, +-1, +-2, ...)
//   VINV_EVEN  x_j = j^2, columns j >= 1 scaled by 1/2
//   VINV_ODD   x_j = (j+1)^2, column j scaled by 1/(2 (j+1))
// With values v(+-i) at a complete symmetric point set, R(x) = E(x^2) + x O(x^2)
// where E(i^2) = (v(i) + v(-i)) / 2 and O(i^2) = (v(i) - v(-i)) / (2 i): the
// EVEN and ODD matrices applied to the sums and differences give E and O.
//   VINV_Q0    x_j = j^4, columns j >= 1 scaled by 1/4
//   VINV_Qt    x_j = (j+1)^4, column j scaled by 1/(4 (j+1)^t)   (t = 1, 2, 3)
// With values v(i^k a) at a complete quartic set, R(x) = sum_t x^t R_t(x^4) and
// sum_k i^(-k t) v(i^k a) = 4 a^t R_t(a^4): the Qt matrices applied to those
// transforms give the R_t.
enum { VINV_GRID = 0, VINV_SYM = 1, VINV_EVEN = 2, VINV_ODD = 3, VINV_Q0 = 4 };
GBR_HD int vinv_point(int mode, int j) {
    return mode == VINV_EVEN ? j * j : mode == VINV_ODD ? (j + 1) * (j + 1) : point_of(mode, j);
}

// one contraction: coefficients (rows of the matrix) x operand (n entries per
// pair and prime, formed from the values according to mode); GEMM_Q0 + t is the
// quarter part R_t of a quartic set (coefficient r of R_t is coefficient 4 r + t)
enum { GEMM_PLAIN = 0, GEMM_EVEN = 1, GEMM_ODD = 2, GEMM_Q0 = 3 };
GBR_HD int gemm_ostride(int mode) { return mode == GEMM_PLAIN ? 1 : mode < GEMM_Q0 ? 2 : 4; }
GBR_HD int gemm_ooff(int mode) { return mode == GEMM_ODD ? 1 : mode >= GEMM_Q0 ? mode - GEMM_Q0 : 0; }
GBR_HD int gemm_vinv_mode(int mode, int sym) {
    return mode == GEMM_EVEN ? VINV_EVEN : mode == GEMM_ODD ? VINV_ODD : mode >= GEMM_Q0 ? VINV_Q0 + mode - GEMM_Q0
         : sym ? VINV_SYM : VINV_GRID;
}
struct GemmGroup {
    const uint32_t *vinv;   // [prime][n][n] inverse Vandermonde matrices
    const uint16_t *vtc;    // the same matrices as bf16 digit tiles (tensor-core path), or null
    int64_t pairs_off;      // the group's pair ids: int32 entries at this byte offset of the plan block
    int32_t n;              // contraction length = matrix size
    int32_t rows;           // coefficients produced (<= n): PLAIN c -> c, EVEN c -> 2c, ODD c -> 2c + 1
    int32_t npairs, mode;
};
struct GemmTile {
    int32_t group, c0, q0, prime;
};
constexpr int kGemmTileM = 64, kGemmTileN = 64;
// tensor-core contraction (gbr_interp_tc.cu): tiles of 64 coefficients x 128 pairs;
// matrices of at most kTcResidentN points run every row tile in one CTA on the
// operand held in shared memory (tile c0 = -1)
constexpr int kTcTileM = 64, kTcTileN = 128, kTcMaxN = 256;
constexpr int kTcResidentChunks = 5, kTcResidentN = 32 * kTcResidentChunks;
size_t vinv_tc_bytes(int n, int rows, int K);
cudaError_t launch_vinv_tc(const uint32_t *vinv, int n, int rows, int K, uint16_t *out, cudaStream_t s);
cudaError_t launch_interp_tc(const ResLaunch &L, const char *planblk, const GemmGroup *groups, const GemmTile *tiles,
                             int ntiles, int xslots, cudaStream_t s);
cudaError_t configure_interp_tc_kernel();
cudaError_t launch_interp_gemm(const ResLaunch &L, const char *planblk, const GemmGroup *groups,
                               const GemmTile *tiles, int ntiles, cudaStream_t s);
cudaError_t launch_zero_init(const ResLaunch &L, cudaStream_t s);

}  // namespace gbr
