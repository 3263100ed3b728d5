// Evaluation and per-(prime, point) resultant (steps A2 + A3 of the path).
//
// One thread per (pair, prime, point) subproblem: the y-coefficients of f and g
// are evaluated at the point (Horner, or even/odd parts at i^2 for the
// symmetric points +-i in lane pairs), then res_{m,n}(F, G) over F_p with the
// formal degrees is computed in shared memory by fraction-free remainder
// steps.  Persistent grid-stride launch per degree bucket.  Each value is
// written as a numerator and a denominator; k_batch_inv forms the quotients.
#include "gbr_device.cuh"
#include "gbr_elim.cuh"

namespace gbr {

// One Horner step acc <- acc a + c on Montgomery residues with c stored as
// c R^2: acc~ a~ + c R^2 = (acc a + c) R^2 < p^2 + p, and one reduction leaves
// (acc a + c) R.
__device__ __forceinline__ uint32_t horner_step(uint32_t acc, uint32_t a, uint32_t c2, const ModP &M) {
    uint32_t lo, hi;
    asm("mad.lo.cc.u32 %0, %2, %3, %4;\n\t"
        "madc.hi.u32 %1, %2, %3, %5;"
        : "=r"(lo), "=r"(hi)
        : "r"(acc), "r"(a), "r"(c2), "r"(0u));
    return mp_redc(lo, hi, M.p, M.pinv);
}

// One Horner step with a fixed multiplier b < p in Shoup's form (bp = floor(b
// 2^32 / p) precomputed): acc b - floor(acc bp / 2^32) p lies in [0, 2p) for any
// 32-bit acc, so with c < p the new accumulator stays below 3p < 2^32 and needs
// no correction inside the loop (three multiply-adds instead of five).  The
// accumulator is congruent to acc b + c modulo p; it is not reduced.
__device__ __forceinline__ uint32_t shoup_step(uint32_t acc, uint32_t b, uint32_t bp, uint32_t c, uint32_t np) {
    return __umulhi(acc, bp) * np + (acc * b + c);
}

// Evaluates rows r0..r0+3 (r0 a multiple of 4) at x = a with four independent
// Horner chains; the residues are laid out [x][row, padded to 4 rows] so the
// four coefficients of one power of x come in one 16-byte load.  Entries past
// a row's degree (and padding rows) are zero, so every chain starts at the
// group's largest degree.  Row r goes to slot (deg - r) of the column.
__device__ __forceinline__ void eval4(const uint32_t *rc, int rows4n, const int32_t *rowdeg, int nrows, int r0,
                                      uint32_t a, const ModP &M, uint32_t *col, int BS) {
    const int nr = min(4, nrows - r0);
    int dmax = -1;
    for (int i = 0; i < nr; ++i) dmax = max(dmax, rowdeg[r0 + i]);
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const uint4 *c = reinterpret_cast<const uint4 *>(rc + r0);
    const int step = rows4n >> 2;
    for (int x = dmax; x >= 0; --x) {
        const uint4 v = c[(int64_t)x * step];
        a0 = horner_step(a0, a, v.x, M);
        a1 = horner_step(a1, a, v.y, M);
        a2 = horner_step(a2, a, v.z, M);
        a3 = horner_step(a3, a, v.w, M);
    }
    const int top = nrows - 1;
    col[(top - r0) * BS] = a0;
    if (nr > 1) col[(top - r0 - 1) * BS] = a1;
    if (nr > 2) col[(top - r0 - 2) * BS] = a2;
    if (nr > 3) col[(top - r0 - 3) * BS] = a3;
}

// Symmetric evaluation of rows r0..r0+3 at +ii and -ii: row(x) = E(x^2) + x O(x^2)
// with E, O the even and odd parts, both evaluated at b = ii^2 (Horner on every
// second coefficient).  The value at this lane's own point goes to its column,
// the value at the partner's point (the opposite sign) to the partner's column.
__device__ __forceinline__ void eval4_sym(const uint32_t *rc, int rows4n, const int32_t *rowdeg, int nrows, int r0,
                                          uint32_t a, uint32_t b, bool negown, const ModP &M, uint32_t *own,
                                          uint32_t *other, int BS) {
    const int nr = min(4, nrows - r0);
    int dmax = -1;
    for (int i = 0; i < nr; ++i) dmax = max(dmax, rowdeg[r0 + i]);
    uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0, o0 = 0, o1 = 0, o2 = 0, o3 = 0;
    const uint4 *c = reinterpret_cast<const uint4 *>(rc + r0);
    const int step = rows4n >> 2;
    int x = dmax;
    if (x >= 0 && (x & 1) == 0) {     // top power even: starts E alone
        const uint4 v = c[(int64_t)x * step];
        e0 = horner_step(0u, b, v.x, M);
        e1 = horner_step(0u, b, v.y, M);
        e2 = horner_step(0u, b, v.z, M);
        e3 = horner_step(0u, b, v.w, M);
        --x;
    }
    for (; x >= 1; x -= 2) {          // x odd: O gets c_x, E gets c_{x-1}
        const uint4 vo = c[(int64_t)x * step];
        const uint4 ve = c[(int64_t)(x - 1) * step];
        o0 = horner_step(o0, b, vo.x, M);
        o1 = horner_step(o1, b, vo.y, M);
        o2 = horner_step(o2, b, vo.z, M);
        o3 = horner_step(o3, b, vo.w, M);
        e0 = horner_step(e0, b, ve.x, M);
        e1 = horner_step(e1, b, ve.y, M);
        e2 = horner_step(e2, b, ve.z, M);
        e3 = horner_step(e3, b, ve.w, M);
    }
    const uint32_t ev[4] = {e0, e1, e2, e3}, ov[4] = {o0, o1, o2, o3};
    const int top = nrows - 1;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (t < nr) {
            const uint32_t io = mp_mul(a, ov[t], M);
            const uint32_t plus = mp_add(ev[t], io, M.p), minus = mp_sub(ev[t], io, M.p);
            const int slot = (top - r0 - t) * BS;
            own[slot] = negown ? minus : plus;
            other[slot] = negown ? plus : minus;
        }
    }
}

// ------------------------------------------------------------------ A2 + A3: evaluate and solve

// One (pair, prime, point) item of a work list on shared-memory columns Fs, Gs
// (stride BS).  Symmetric pairs need the whole warp: lane l and lane l ^ 16
// hand each other values.
__device__ __forceinline__ void evalres_item(const ResLaunch &L, const WorkList &w, int64_t item, uint32_t *Fs,
                                             uint32_t *Gs, int BS) {
    int bi = wl_find(w.start, w.n, item);
    int q = w.pairs[bi];
    int64_t local = item - w.start[bi];
    const PairPlan &P = L.plan[q];
    const int rf4 = rows4(P.m), rg4 = rows4(P.n);
    const int32_t *dgf = L.rowdeg + P.rowdeg_f;
    const int32_t *dgg = L.rowdeg + P.rowdeg_g;
    if (P.sym) {
        // lanes 0-15 take points +a, lanes 16-31 take -a (same a); a lane
        // evaluates even and odd parts of one polynomial at a^2 and hands the
        // partner its value: f-lanes do f, g-lanes do g.  a = ii (PTS_SYM) or
        // u^ii (PTS_ROOTS, -u^ii = u^(ii + Pe/2))
        const bool roots = P.sym == PTS_ROOTS, quad = P.sym == PTS_QUAD;
        const int per = P.tiles * 32;      // lanes per prime (a quartic set's warps span its primes)
        int i = quad ? 0 : (int)(local / per);
        const int r = quad ? (int)(local & 31) : (int)(local % per);
        const int lane = r & 31;
        const int ii = (r >> 5) * 16 + (lane & 15);
        const bool glane = lane >= 16;
        QuadLane ql{0, 0, false};
        if (quad) {
            // lane pair l = 2 qi + k0 of the warp takes x = i^k0 a of quadruple qi, its
            // partner -x = i^(k0+2) a
            ql = quad_lane(P.P, P.k, local >> 5, (lane & 15) >> 1);
            i = ql.i;
        }
        const int pidx = prime_of(P, L.pmap, i);
        const ModP M = L.mods[pidx];
        int j;
        uint32_t a;   // this lane pair's point x (Montgomery form); lanes 16-31 take -x
        if (roots) {
            j = ii < P.Pe / 2 ? (glane ? ii + P.Pe / 2 : ii) : -1;
            a = root_pow(L.roots + (int64_t)pidx * kRootTabWords, (ii * (kRootOrder / P.Pe)) & (kRootOrder - 1), M);
        } else if (quad) {
            const int k0 = lane & 1;
            j = quad_index(ql, k0 + (glane ? 2 : 0));
            const uint32_t im = iota_mont(L, pidx);
            a = mp_to((uint32_t)ql.a, M);
            if (k0) a = mp_mul(a, im, M);
        } else {
            j = ii == 0 ? (glane ? -1 : 0) : (glane ? 2 * ii : 2 * ii - 1);
            a = mp_to((uint32_t)ii, M);
        }
        const uint32_t b = mp_mul(a, a, M);
        const uint32_t *rbase = L.res + P.res_off + (int64_t)i * P.S;
        const uint32_t *rc = glane ? rbase + (int64_t)(P.dxf + 1) * rf4 : rbase;
        const int32_t *dg = glane ? dgg : dgf;
        const int nrows = (glane ? P.n : P.m) + 1;
        const int r4 = glane ? rg4 : rf4;
        uint32_t *own = (glane ? Gs : Fs);
        uint32_t *other = own + (glane ? -16 : 16);
        for (int r0 = 0; r0 < nrows; r0 += 4) eval4_sym(rc, r4, dg, nrows, r0, a, b, glane, M, own, other, BS);
        __syncwarp();
        if (j >= 0 && j < P.Pe) {
            L.val[P.val_off + (int64_t)i * P.Pe + j] = res_formal(Fs, P.m, Gs, P.n, BS, M);
            L.den[P.val_off + (int64_t)i * P.Pe + j] = M.r1;
        }
        __syncwarp();
        return;
    }
    int i = (int)(local / P.Pe);
    int j = (int)(local % P.Pe);
    const ModP M = L.mods[prime_of(P, L.pmap, i)];
    const uint32_t a = mp_to((uint32_t)j, M);
    const uint32_t *rf = L.res + P.res_off + (int64_t)i * P.S;
    const uint32_t *rg = rf + (int64_t)(P.dxf + 1) * rf4;
    for (int r0 = 0; r0 <= P.m; r0 += 4) eval4(rf, rf4, dgf, P.m + 1, r0, a, M, Fs, BS);
    for (int r0 = 0; r0 <= P.n; r0 += 4) eval4(rg, rg4, dgg, P.n + 1, r0, a, M, Gs, BS);
    if (P.flag_off >= 0) {
        // a point where a leading coefficient vanishes is unlucky: flag it, so
        // interpolation takes the spare points instead (its formal-degree value
        // below is still exact)
        const uint8_t unlucky = Fs[0] == 0u || Gs[0] == 0u;
        L.pflags[P.flag_off + (int64_t)i * P.Pe + j] = unlucky;
        if (unlucky) atomicAdd(L.dropped, 1ull);
    }
    L.val[P.val_off + (int64_t)i * P.Pe + j] = res_formal(Fs, P.m, Gs, P.n, BS, M);
    L.den[P.val_off + (int64_t)i * P.Pe + j] = M.r1;
}

__global__ void k_evalres(ResLaunch L, WorkList w, int SF, int SG) {
    if (stage_skipped(L)) return;
    extern __shared__ uint32_t smem[];
    const int BS = blockDim.x;
    uint32_t *Fs = smem + threadIdx.x;
    uint32_t *Gs = smem + SF * BS + threadIdx.x;
    for (int64_t item = blockIdx.x * (int64_t)BS + threadIdx.x; item < w.total; item += (int64_t)gridDim.x * BS)
        evalres_item(L, w, item, Fs, Gs, BS);
}

// Symmetric pairs of shape (N, N), (N, N-1) or (N-1, N): the same lane pairs
// as k_evalres (or, on the quartic set, quadruples of lanes evaluating in radix
// 4), but the evaluated columns stay in registers (handed across by shuffles or
// the warp's exchange buffer) and res_chain solves in registers.  A warp with a lane whose
// subproblem needs the general solver is appended to `redo` and written by
// k_evalres_redo instead (whole warps, since lane pairs share evaluations).
// blocks of 256 per SM the register allocation must allow: three (80 registers,
// a few spills to L1)
// measured fastest at N = 20 (12.0 against 12.5 ms with 128 registers on the
// 4096-pair degree-20 batch); larger N need more registers than that
constexpr int reg_min_blocks(int N) { return N <= 20 ? 3 : N <= 27 ? 2 : 1; }

// Quartic set, radix 4: lane 8 role + qi of the warp takes the point i^role a of
// quadruple qi (quad_lane).  The four lanes of a quadruple evaluate 4-row chunks of
// f and g at all four of its points at once: with c = a^4 a row is
// P_0(c) + x P_1(c) + x^2 P_2(c) + x^3 P_3(c) at x = i^k a, P_t its part of the
// powers x^(4 s + t), each by Shoup steps at c on the stored c R^2 residues.  Slot s
// holds the chunk positions f 2s, g 2s, f 2s+1, g 2s+1, taken by roles 0..3 (s even)
// or 3..0 (s odd), which evens out the shorter rows of total-degree inputs.  The
// values meet in the warp's exchange buffer (per position, row and quadruple the
// four points), where each lane picks those at its own point.
template <int N>
__device__ __forceinline__ void quad_eval4(const ResLaunch &L, const PairPlan &P, int64_t local, int lane, uint4 *xb,
                                           uint32_t (&F)[N + 1], uint32_t (&G)[N + 1], int &i, int &j, ModP &M) {
    const int role = lane >> 3, qi = lane & 7;
    const QuadLane ql = quad_lane(P.P, P.k, local >> 5, qi);
    i = ql.i;
    j = quad_index(ql, role);
    const int pidx = prime_of(P, L.pmap, i);
    M = L.mods[pidx];
    const uint32_t im = iota_mont(L, pidx);   // i R
    // powers of a in normal form (a <= 4096, so a^2 < 2^24 < p)
    const uint32_t a1 = (uint32_t)ql.a, a2 = a1 * a1;
    const uint32_t a3 = mp_mul(mp_mul(a2, a1, M), M.r2, M), a4 = mp_mul(mp_mul(a2, a2, M), M.r2, M);
    const uint32_t c4p = (uint32_t)(((uint64_t)a4 << 32) / M.p);
    const uint32_t np = 0u - M.p;
    const uint32_t *rf = L.res + P.res_off + (int64_t)i * P.S;
    const uint32_t *rg = rf + (int64_t)(P.dxf + 1) * rows4(P.m);
    const uint32_t *xw = reinterpret_cast<const uint32_t *>(xb);
    constexpr int CF = (N + 1 + 3) / 4;    // 4-row chunks of one polynomial, at most
    constexpr int SL = (2 * CF + 3) / 4;   // slots of four chunks
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int pos = (s & 1) ? 3 - role : role;
        const bool gp = pos & 1;
        const int c = 2 * s + (pos >> 1), r0 = 4 * c;
        const int nrows = (gp ? P.n : P.m) + 1;
        uint32_t e[4][4];   // [part t][row of the chunk]: R^2 P_t(c), below 3p
#pragma unroll
        for (int t = 0; t < 4; ++t) e[t][0] = e[t][1] = e[t][2] = e[t][3] = 0u;
        if (c < CF && r0 < nrows) {
            const int32_t *dg = L.rowdeg + (gp ? P.rowdeg_g : P.rowdeg_f);
            const int step = rows4(gp ? P.n : P.m) >> 2;
            const uint4 *cp = reinterpret_cast<const uint4 *>((gp ? rg : rf) + r0);
            int dmax = -1;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (r0 + t < nrows) dmax = max(dmax, dg[r0 + t]);
            if (dmax >= 0) {
                int g = dmax >> 2;   // top group of four powers: only those up to dmax
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (4 * g + t <= dmax) {
                        const uint4 v = cp[(int64_t)(4 * g + t) * step];
                        e[t][0] = v.x;
                        e[t][1] = v.y;
                        e[t][2] = v.z;
                        e[t][3] = v.w;
                    }
                for (--g; g >= 0; --g) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const uint4 v = cp[(int64_t)(4 * g + t) * step];
                        e[t][0] = shoup_step(e[t][0], a4, c4p, v.x, np);
                        e[t][1] = shoup_step(e[t][1], a4, c4p, v.y, np);
                        e[t][2] = shoup_step(e[t][2], a4, c4p, v.z, np);
                        e[t][3] = shoup_step(e[t][3], a4, c4p, v.w, np);
                    }
                }
            }
        }
        // the row at x = a, i a, -a, -i a (R-form, below p): with A_t = a^t P_t,
        // (P_0 + A_2) +- (A_1 + A_3) and (P_0 - A_2) +- i (A_1 - A_3)
        uint4 out[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t p0 = mp_redc(e[0][q], 0u, M.p, M.pinv);
            const uint32_t A1 = mp_mul(e[1][q], a1, M), A2 = mp_mul(e[2][q], a2, M), A3 = mp_mul(e[3][q], a3, M);
            const uint32_t u = mp_add(p0, A2, M.p), v = mp_sub(p0, A2, M.p);
            const uint32_t sm = mp_add(A1, A3, M.p), d = mp_mul(mp_sub(A1, A3, M.p), im, M);
            out[q] = make_uint4(mp_add(u, sm, M.p), mp_add(v, d, M.p), mp_sub(u, sm, M.p), mp_sub(v, d, M.p));
        }
        __syncwarp();   // the previous slot's reads are done
#pragma unroll
        for (int q = 0; q < 4; ++q) xb[(pos * 4 + q) * 8 + qi] = out[q];
        __syncwarp();
#pragma unroll
        for (int ps = 0; ps < 4; ++ps) {
            const int cc = 2 * s + (ps >> 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = 4 * cc + q;
                if (row <= N) {
                    const uint32_t v = xw[((ps * 4 + q) * 8 + qi) * 4 + role];
                    if (ps & 1) G[row] = v;
                    else F[row] = v;
                }
            }
        }
    }
}

// Integer points and roots of unity in +-a lane pairs: lane l < 16 and its partner
// l + 16 take a and -a; the f-lane evaluates f's rows, the g-lane g's, each at both
// points from the even and odd parts at a^2, and they hand each other the values.
template <int N>
__device__ __forceinline__ void pair_eval(const ResLaunch &L, const PairPlan &P, int64_t local, int lane,
                                          uint32_t (&F)[N + 1], uint32_t (&G)[N + 1], int &i, int &j, ModP &M) {
    const int per = P.tiles * 32;
    i = (int)(local / per);
    const int r = (int)(local % per);
    const int ii = (r >> 5) * 16 + (lane & 15);
    const bool glane = lane >= 16;
    const bool roots = P.sym == PTS_ROOTS;   // warp-uniform: a warp is one (pair, prime, tile)
    const int pidx = prime_of(P, L.pmap, i);
    M = L.mods[pidx];
    // the point a in normal form: ii (PTS_SYM), or u^ii for the primitive Pe-th root
    // of unity u = w^(2^kRootLog / Pe) (PTS_ROOTS; the partner lane's point -a is
    // u^(ii + Pe/2))
    j = ii == 0 ? (glane ? -1 : 0) : (glane ? 2 * ii : 2 * ii - 1);
    uint32_t a = (uint32_t)ii, b = (uint32_t)ii * (uint32_t)ii;
    if (roots) {
        j = ii < P.Pe / 2 ? (glane ? ii + P.Pe / 2 : ii) : -1;
        a = mp_from(root_pow(L.roots + (int64_t)pidx * kRootTabWords, (ii * (kRootOrder / P.Pe)) & (kRootOrder - 1),
                             M),
                    M);
        b = mp_mul(mp_mul(a, a, M), M.r2, M);
    }
    // even and odd parts at b = a^2 (below p) by Shoup steps on the stored
    // c R^2 residues, so the parts come out as R^2 E and R^2 O
    const uint32_t bp = (uint32_t)(((uint64_t)b << 32) / M.p);
    const uint32_t np = 0u - M.p;
    const int rf4 = rows4(P.m);
    const uint32_t *rbase = L.res + P.res_off + (int64_t)i * P.S;
    const uint32_t *rc = glane ? rbase + (int64_t)(P.dxf + 1) * rf4 : rbase;
    const int32_t *dg = L.rowdeg + (glane ? P.rowdeg_g : P.rowdeg_f);
    const int nrows = (glane ? P.n : P.m) + 1;
    const int step = (glane ? rows4(P.n) : rf4) >> 2;
    // own[k]: this lane's polynomial at its own point; oth[k]: at the partner's
    uint32_t own[N + 1], oth[N + 1];
#pragma unroll
    for (int r0 = 0; r0 <= N; r0 += 4) {
        uint32_t e[4] = {0u, 0u, 0u, 0u}, o[4] = {0u, 0u, 0u, 0u};
        if (r0 < nrows) {
            int dmax = -1;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (r0 + t < nrows) dmax = max(dmax, dg[r0 + t]);
            const uint4 *c = reinterpret_cast<const uint4 *>(rc + r0);
            int x = dmax;
            if (x >= 0 && (x & 1) == 0) {
                const uint4 v = c[(int64_t)x * step];
                e[0] = v.x;
                e[1] = v.y;
                e[2] = v.z;
                e[3] = v.w;
                --x;
            }
            for (; x >= 1; x -= 2) {
                const uint4 vo = c[(int64_t)x * step];
                const uint4 ve = c[(int64_t)(x - 1) * step];
                o[0] = shoup_step(o[0], b, bp, vo.x, np);
                o[1] = shoup_step(o[1], b, bp, vo.y, np);
                o[2] = shoup_step(o[2], b, bp, vo.z, np);
                o[3] = shoup_step(o[3], b, bp, vo.w, np);
                e[0] = shoup_step(e[0], b, bp, ve.x, np);
                e[1] = shoup_step(e[1], b, bp, ve.y, np);
                e[2] = shoup_step(e[2], b, bp, ve.z, np);
                e[3] = shoup_step(e[3], b, bp, ve.w, np);
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (r0 + t <= N) {
                // R E = redc(R^2 E); R a O = redc(R^2 O a) (R^2 O < 3p, so
                // both inputs stay below p 2^32)
                const uint32_t ev = mp_redc(e[t], 0u, M.p, M.pinv);
                const uint32_t io = mp_mul(o[t], a, M);
                const uint32_t plus = mp_add(ev, io, M.p), minus = mp_sub(ev, io, M.p);
                own[r0 + t] = glane ? minus : plus;
                oth[r0 + t] = glane ? plus : minus;
            }
        }
    }
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        const uint32_t got = __shfl_xor_sync(0xffffffffu, oth[k], 16);
        F[k] = glane ? got : own[k];
        G[k] = glane ? own[k] : got;
    }
}

template <int N>
__global__ void __launch_bounds__(256, reg_min_blocks(N)) k_evalres_reg(ResLaunch L, WorkList w, unsigned long long *redo_n,
                                                     int64_t *redo) {
    if (stage_skipped(L)) return;
    __shared__ uint4 xq[256 / 32][4 * 4 * 8];   // per warp: the quartic exchange buffer
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < w.total;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int bi = wl_find(w.start, w.n, item);
        const int q = w.pairs[bi];
        const int64_t local = item - w.start[bi];
        const PairPlan &P = L.plan[q];
        const int lane = (int)(local & 31);   // a pair's lanes start at a multiple of 32
        uint32_t F[N + 1], G[N + 1];
        int i, j;
        ModP M;
        // warp-uniform: a warp is within one pair
        if (P.sym == PTS_QUAD) quad_eval4<N>(L, P, local, lane, xq[threadIdx.x >> 5], F, G, i, j, M);
        else pair_eval<N>(L, P, local, lane, F, G, i, j, M);
        bool ok;
        uint32_t den;
        const uint32_t v = res_chain_frac<N>(F, G, P.m, P.n, M, ok, den);
        const bool valid = j >= 0 && j < P.Pe;
        if (__ballot_sync(0xffffffffu, valid && !ok)) {
            if (lane == 0) redo[atomicAdd(redo_n, 1ull)] = item;
        } else if (valid) {
            // the quotient v / den: k_batch_inv divides once the whole segment is in
            L.val[P.val_off + (int64_t)i * P.Pe + j] = v;
            L.den[P.val_off + (int64_t)i * P.Pe + j] = den;
        }
    }
}

// The warps listed by k_evalres_reg, solved on shared-memory columns.
__global__ void k_evalres_redo(ResLaunch L, WorkList w, int SF, const unsigned long long *redo_n,
                               const int64_t *redo) {
    if (stage_skipped(L)) return;
    extern __shared__ uint32_t smem[];
    const int BS = blockDim.x;
    uint32_t *Fs = smem + threadIdx.x;
    uint32_t *Gs = smem + SF * BS + threadIdx.x;
    const int64_t nw = (int64_t)*redo_n;
    const int lane = threadIdx.x & 31;
    for (int64_t e = (blockIdx.x * (int64_t)BS + threadIdx.x) >> 5; e < nw; e += ((int64_t)gridDim.x * BS) >> 5)
        evalres_item(L, w, redo[e] + lane, Fs, Gs, BS);
}

// The quotients of the register form (written as numerator and denominator by
// k_evalres_reg): one warp per (pair, prime, segment of kInvSeg values), Montgomery's
// batch inversion - the prefix products of the segment's denominators, one Fermat
// inverse of their product, then every inverse from a prefix and a suffix - so
// that a segment pays about four products per value instead of one inverse each.
// Entries written by the other evaluation kernels carry the denominator 1 (R in
// Montgomery form).
constexpr int kInvSeg = kInvSegment;   // values per warp: 16 per lane, interleaved for coalescing

__global__ void __launch_bounds__(256) k_batch_inv(ResLaunch L, WorkList w) {
    if (stage_skipped(L)) return;
    const int lane = threadIdx.x & 31;
    for (int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; item < w.total;
         item += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int bi = wl_find(w.start, w.n, item);
        const PairPlan &P = L.plan[w.pairs[bi]];
        const int64_t local = item - w.start[bi];
        const int nseg = (P.Pe + kInvSeg - 1) / kInvSeg;
        const int i = (int)(local / nseg), sg = (int)(local % nseg);
        const ModP M = L.mods[prime_of(P, L.pmap, i)];
        const int64_t base = P.val_off + (int64_t)i * P.Pe + (int64_t)sg * kInvSeg;
        const int cnt = min(kInvSeg, P.Pe - sg * kInvSeg);
        uint32_t d[kInvSeg / 32], pre[kInvSeg / 32];
        uint32_t run = M.r1;
#pragma unroll
        for (int u = 0; u < kInvSeg / 32; ++u) {
            const int t = u * 32 + lane;
            d[u] = t < cnt ? L.den[base + t] : M.r1;
            run = mp_mul(run, d[u], M);
            pre[u] = run;   // d[0] ... d[u]
        }
        // products of the lanes' runs: inclusive prefix, suffix, and the whole segment
        uint32_t incl = run, suf = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a = __shfl_up_sync(0xffffffffu, incl, o);
            const uint32_t b = __shfl_down_sync(0xffffffffu, suf, o);
            if (lane >= o) incl = mp_mul(incl, a, M);
            if (lane + o < 32) suf = mp_mul(suf, b, M);
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t before = __shfl_up_sync(0xffffffffu, incl, 1);
        uint32_t after = __shfl_down_sync(0xffffffffu, suf, 1);
        if (lane == 0) before = M.r1;
        if (lane == 31) after = M.r1;
        // 1 / (this lane's run) = (1 / total) (runs of the other lanes)
        uint32_t inv = mp_mul(mp_mul(mp_inv(total, M), before, M), after, M);
#pragma unroll
        for (int u = kInvSeg / 32 - 1; u >= 0; --u) {
            const int t = u * 32 + lane;
            const uint32_t id = u > 0 ? mp_mul(inv, pre[u - 1], M) : inv;   // 1 / d[u]
            if (t < cnt) L.val[base + t] = mp_mul(L.val[base + t], id, M);
            inv = mp_mul(inv, d[u], M);
        }
    }
}

cudaError_t launch_batch_inv(const ResLaunch &L, const WorkList &w, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    const int block = 256;
    const int grid = persistent_grid(k_batch_inv, block, 0, (w.total * 32 + block - 1) / block);
    k_batch_inv<<<grid, block, 0, s>>>(L, w);
    return cudaGetLastError();
}

cudaError_t launch_evalres(const ResLaunch &L, const WorkList &w, int SF, int SG, int block, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    size_t smem = (size_t)(SF + SG) * block * sizeof(uint32_t);
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    int grid = persistent_grid(k_evalres, block, smem, (w.total + block - 1) / block);
    k_evalres<<<grid, block, smem, s>>>(L, w, SF, SG);
    return cudaGetLastError();
}


using RegKernel = void (*)(ResLaunch, WorkList, unsigned long long *, int64_t *);

static RegKernel reg_kernel(int N) {
    switch (N) {
#define GBR_REG_CASE(n) \
    case n:             \
        return k_evalres_reg<n>;
        GBR_REG_CASE(2) GBR_REG_CASE(3) GBR_REG_CASE(4) GBR_REG_CASE(5) GBR_REG_CASE(6) GBR_REG_CASE(7)
        GBR_REG_CASE(8) GBR_REG_CASE(9) GBR_REG_CASE(10) GBR_REG_CASE(11) GBR_REG_CASE(12) GBR_REG_CASE(13)
        GBR_REG_CASE(14) GBR_REG_CASE(15) GBR_REG_CASE(16) GBR_REG_CASE(17) GBR_REG_CASE(18) GBR_REG_CASE(19)
        GBR_REG_CASE(20) GBR_REG_CASE(21) GBR_REG_CASE(22) GBR_REG_CASE(23) GBR_REG_CASE(24) GBR_REG_CASE(25)
        GBR_REG_CASE(26) GBR_REG_CASE(27) GBR_REG_CASE(28) GBR_REG_CASE(29) GBR_REG_CASE(30) GBR_REG_CASE(31)
        GBR_REG_CASE(32)
#undef GBR_REG_CASE
    }
    return nullptr;
}
static_assert(kRegMinN == 2 && kRegMaxN == 32, "reg_kernel covers kRegMinN..kRegMaxN");

cudaError_t launch_evalres_reg(const ResLaunch &L, const WorkList &w, int N, int block, unsigned long long *redo_n,
                               int64_t *redo, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    RegKernel k = reg_kernel(N);
    if (!k || w.total % 32 != 0 || block % 32 != 0) return cudaErrorInvalidValue;
    int grid = persistent_grid(k, block, 0, (w.total + block - 1) / block);
    k<<<grid, block, 0, s>>>(L, w, redo_n, redo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the redo pass reads its count on the device; with nothing listed its
    // blocks return at once
    const int rb = 128, SF = (N + 1 + 3) / 4 * 4;
    const size_t smem = (size_t)2 * SF * rb * sizeof(uint32_t);
    grid = persistent_grid(k_evalres_redo, rb, smem, (w.total / 32 + rb / 32 - 1) / (rb / 32));
    k_evalres_redo<<<grid, rb, smem, s>>>(L, w, SF, redo_n, redo);
    return cudaGetLastError();
}

cudaError_t configure_evalres_kernel() {
    cudaError_t e = cudaFuncSetAttribute(k_evalres_redo, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_evalres, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

}  // namespace gbr
