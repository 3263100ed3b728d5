// Evaluation and per-(prime, point) resultant (steps A2 + A3 of the path).
//
// One thread per (pair, prime, point) subproblem: the y-coefficients of f and g
// are evaluated at the point (Horner, or even/odd parts at i^2 for the
// symmetric points +-i in lane pairs), then res_{m,n}(F, G) over F_p with the
// formal degrees is computed in shared memory by fraction-free remainder
// steps.  Persistent grid-stride launch per degree bucket.
#include "gbr_device.cuh"

namespace gbr {

// ------------------------------------------------------------------ A3: resultant mod p

// res_{da,db}(A, B) over F_p with formal degrees.  A and B live in shared memory,
// one column per thread (stride BS); A[t*BS] is the coefficient of y^(da - t).
// Identities used (lc = leading coefficient):
//   res_{a,b}(A,B) = (-1)^{ab} res_{b,a}(B,A)
//   lc(A) != 0:  res_{a,b}(A,B) = lc(A)^{b-b'} res_{a,b'}(A,B')   (B' = B without zero top terms)
//   lc(B) = zeta != 0, R = A mod B, deg R = r:
//       res_{a,b}(A,B) = (-1)^{ab} zeta^{a-r} res_{b,r}(B,R)
//   res_{b,r}(B, c R) = c^b res_{b,r}(B,R)    (R is reached as zeta^e R by e fraction-free steps)
//   res_{a,0}(A, b0) = b0^a ; res_{0,0} = 1 ; both leading coefficients zero -> 0.
//
// Normal rounds (deg A = deg B + 1 = d + 1) are done in one pass:
//   zeta^2 A - (zeta alpha x + q0) B,  q0 = zeta a_d - alpha b_{d-1},
// three products per coefficient and one reduction (mp_fma3).  Such a round
// contributes zeta^(2d) to the divisor and zeta^2 to the multiplier, i.e. a net
// Z^(d-1) with Z = zeta^2 in the divisor.  These are collected without powers:
// Q holds the product of the Z of all normal rounds so far, and whenever the
// divisor degree drops by delta between rounds, D *= Q^delta (delta is 1 in the
// normal case); after the last round D *= Q^(d_last - 1).  Each Z_r then appears
// in D with exponent (d_r - d_last) + (d_last - 1) = d_r - 1.  Other rounds keep
// explicit powers.
GBR_HD uint32_t res_formal(uint32_t *A, int da, uint32_t *B, int db, int BS, const ModP &M) {
    const uint32_t one = M.r1;
    uint32_t acc = one, den = one, Q = one, D = one;
    int prev_db = -1;
    bool neg = false;
    if (da == 0 && db == 0) return one;
    if (A[0] == 0 && B[0] == 0) return 0u;
    if (A[0] == 0) {
        int da0 = da;
        while (da >= 0 && A[0] == 0) { A += BS; --da; }
        if ((da0 * db) & 1) neg = !neg;
        if (da < 0) {
            if (db >= 1) return 0u;
            return mp_pow(B[0], (uint32_t)da0, M);
        }
        acc = mp_pow(B[0], (uint32_t)(da0 - da), M);
        uint32_t *t = A; A = B; B = t;
        int ti = da; da = db; db = ti;
    } else if (B[0] == 0) {
        int db0 = db;
        while (db >= 0 && B[0] == 0) { B += BS; --db; }
        if (db < 0) {
            if (da >= 1) return 0u;
            return mp_pow(A[0], (uint32_t)db0, M);
        }
        acc = mp_pow(A[0], (uint32_t)(db0 - db), M);
    }
    while (true) {
        if (da < db) {
            uint32_t *t = A; A = B; B = t;
            int ti = da; da = db; db = ti;
            if ((da * db) & 1) neg = !neg;
        }
        if (db == 0) {
            acc = mp_mul(acc, mp_pow(B[0], (uint32_t)da, M), M);
            break;
        }
        if (prev_db >= 0) D = mp_mul(D, prev_db - db == 1 ? Q : mp_pow(Q, (uint32_t)(prev_db - db), M), M);
        prev_db = db;
        const uint32_t zeta = B[0];
        if (da == db + 1) {
            const uint32_t alpha = A[0];
            const uint32_t z2 = mp_mul(zeta, zeta, M);
            const uint32_t nza = M.p - mp_mul(zeta, alpha, M);
            const uint32_t nq0 = M.p - mp_mulsub(zeta, A[BS], alpha, B[BS], M);
            // new A[s] = z2 A[s+2] - (zeta alpha) B[s+2] - q0 B[s+1], s = 0..db-1, B[db+1] = 0
            int s = 0;
            for (; s + 4 <= db; s += 4) {
                uint32_t x0 = A[(s + 2) * BS], x1 = A[(s + 3) * BS], x2 = A[(s + 4) * BS], x3 = A[(s + 5) * BS];
                uint32_t b1 = B[(s + 1) * BS], b2 = B[(s + 2) * BS], b3 = B[(s + 3) * BS], b4 = B[(s + 4) * BS];
                uint32_t b5 = s + 5 <= db ? B[(s + 5) * BS] : 0u;
                uint32_t r0 = mp_fma3(z2, x0, nza, b2, nq0, b1, M);
                uint32_t r1 = mp_fma3(z2, x1, nza, b3, nq0, b2, M);
                uint32_t r2 = mp_fma3(z2, x2, nza, b4, nq0, b3, M);
                uint32_t r3 = mp_fma3(z2, x3, nza, b5, nq0, b4, M);
                A[(s + 2) * BS] = r0;
                A[(s + 3) * BS] = r1;
                A[(s + 4) * BS] = r2;
                A[(s + 5) * BS] = r3;
            }
            for (; s < db; ++s) {
                uint32_t b2 = s + 2 <= db ? B[(s + 2) * BS] : 0u;
                A[(s + 2) * BS] = mp_fma3(z2, A[(s + 2) * BS], nza, b2, nq0, B[(s + 1) * BS], M);
            }
            A += 2 * BS;
            da = db - 1;
            while (da >= 0 && A[0] == 0) { A += BS; --da; }
            if (da < 0) return 0u;
            Q = mp_mul(Q, z2, M);
            if (da < db - 1) acc = mp_mul(acc, mp_pow(zeta, (uint32_t)(db - 1 - da), M), M);
        } else {
            const int DA = da;
            int e = 0;
            while (da >= db) {
                const uint32_t q = A[0];
                int t = 1;
                for (; t <= db; ++t) A[t * BS] = mp_mulsub(zeta, A[t * BS], q, B[t * BS], M);
                for (; t <= da; ++t) A[t * BS] = mp_mul(zeta, A[t * BS], M);
                A += BS;
                --da;
                ++e;
                while (da >= 0 && A[0] == 0) { A += BS; --da; }
            }
            if (da < 0) return 0u;
            if ((DA * db) & 1) neg = !neg;
            acc = mp_mul(acc, mp_pow(zeta, (uint32_t)(DA - da), M), M);
            den = mp_mul(den, mp_pow(zeta, (uint32_t)(e * db), M), M);
        }
        uint32_t *t = A; A = B; B = t;
        int ti = da; da = db; db = ti;
    }
    if (prev_db >= 1) D = mp_mul(D, mp_pow(Q, (uint32_t)(prev_db - 1), M), M);
    den = mp_mul(den, D, M);
    uint32_t r = mp_mul(acc, mp_inv(den, M), M);
    return neg ? mp_neg(r, M.p) : r;
}

// Register form of res_formal for the shapes (N, N), (N, N-1) and (N-1, N) when
// the remainder sequence is normal at this point (every remainder has degree
// one less than its divisor) -- the generic case.  F[k], G[k] hold the
// coefficients of y^k.  Degrees are compile-time constants in every round, so
// the polynomials stay in registers.  Returns with ok = false when a leading
// coefficient vanishes at the point or the sequence is not normal (the caller
// then solves the subproblem with res_formal); a remainder that vanishes
// identically proves a common factor of positive degree and gives 0.
//   (N-1, N): res_{N-1,N}(F,G) = res_{N,N-1}(G,F), since (N-1) N is even.
//   (N, N):   with alpha = lc A, zeta = lc B and B' = alpha B - zeta A,
//             res_{N,N}(A,B) = alpha^(1-N) res_{N,N-1}(A,B') (the remainder
//             identity applied to res(B, A), whose sign cancels the swap's).
//   Normal rounds are the fused three-product rounds of res_formal with the
//   same telescoped divisor D = Q_0 Q_1 ... (Q_t = Z_0 ... Z_t, Z = zeta^2).
template <int N>
GBR_HD void chain_round(uint32_t (&U)[N + 1], const uint32_t (&V)[N + 1], const int d, const bool first,
                        uint32_t &Dq, uint32_t &Q, bool &done, bool &ok, const ModP &M) {
    // U has degree d + 1, V degree d; U <- zeta^2 U - (zeta alpha y + q0) V
    if (done) return;
    const uint32_t zeta = V[d], alpha = U[d + 1];
    if (!first) Dq = mp_mul(Dq, Q, M);
    const uint32_t z2 = mp_mul(zeta, zeta, M);
    const uint32_t nza = M.p - mp_mul(zeta, alpha, M);
    const uint32_t nq0 = M.p - mp_mulsub(zeta, U[d], alpha, V[d - 1], M);
    U[0] = mp_fma2(z2, U[0], nq0, V[0], M);
#pragma unroll
    for (int k = 1; k < d; ++k) U[k] = mp_fma3(z2, U[k], nza, V[k - 1], nq0, V[k], M);
    Q = mp_mul(Q, z2, M);
    if (U[d - 1] == 0u) {
        uint32_t any = 0u;
#pragma unroll
        for (int k = 0; k < d - 1; ++k) any |= U[k];
        done = true;
        ok = any == 0u;   // identically zero: the resultant is 0 (Dq is then ignored)
        Dq = 0u;
    }
}

template <int N>
GBR_HD uint32_t res_chain(const uint32_t (&F)[N + 1], const uint32_t (&G)[N + 1], int m, int n, const ModP &M,
                          bool &ok) {
    static_assert(N >= 2, "the register form starts at degree 2");
    const bool sw = m != N;   // (N-1, N): solve res(G, F)
    const int nb = sw ? m : n;
    uint32_t A[N + 1], B[N + 1];
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        A[k] = sw ? G[k] : F[k];
        B[k] = sw ? F[k] : G[k];
    }
    ok = false;
    // (a constant index keeps B in registers)
    if (A[N] == 0u || (nb == N ? B[N] : B[N - 1]) == 0u) return 0u;   // a leading coefficient vanishes here
    uint32_t acc = M.r1, den = M.r1, Dq = M.r1, Q = M.r1;
    if (nb == N) {
        const uint32_t alpha = A[N], zeta = B[N];
        uint32_t any = 0u;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            B[k] = mp_mulsub(alpha, B[k], zeta, A[k], M);
            any |= B[k];
        }
        if (B[N - 1] == 0u) {
            ok = any == 0u;
            return 0u;
        }
        acc = alpha;
        den = mp_pow(alpha, (uint32_t)N, M);
    }
    bool done = false;
    ok = true;
#pragma unroll
    for (int t = 0; t < N - 1; t += 2) {
        chain_round<N>(A, B, N - 1 - t, t == 0, Dq, Q, done, ok, M);
        if (t + 1 < N - 1) chain_round<N>(B, A, N - 2 - t, false, Dq, Q, done, ok, M);
    }
    if (done) return 0u;   // ok tells a zero resultant from a sequence that is not normal
    const uint32_t c = ((N - 2) % 2 == 0) ? A[0] : B[0];   // the last remainder, a constant
    acc = mp_mul(acc, c, M);
    den = mp_mul(den, Dq, M);
    return mp_mul(acc, mp_inv(den, M), M);
}

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
        // lanes 0-15 take points +ii, lanes 16-31 take -ii (same ii); a lane
        // evaluates even and odd parts of one polynomial at ii^2 and hands the
        // partner its value: f-lanes do f, g-lanes do g
        const int per = P.tiles * 32;
        const int i = (int)(local / per);
        const int r = (int)(local % per);
        const int lane = r & 31;
        const int ii = (r >> 5) * 16 + (lane & 15);
        const bool glane = lane >= 16;
        const int j = ii == 0 ? (glane ? -1 : 0) : (glane ? 2 * ii : 2 * ii - 1);
        const ModP M = L.mods[prime_of(P, L.pmap, i)];
        const uint32_t a = mp_to((uint32_t)ii, M);
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
        if (j >= 0 && j < P.Pe) L.val[P.val_off + (int64_t)i * P.Pe + j] = res_formal(Fs, P.m, Gs, P.n, BS, M);
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
}

__global__ void k_evalres(ResLaunch L, WorkList w, int SF, int SG) {
    extern __shared__ uint32_t smem[];
    const int BS = blockDim.x;
    uint32_t *Fs = smem + threadIdx.x;
    uint32_t *Gs = smem + SF * BS + threadIdx.x;
    for (int64_t item = blockIdx.x * (int64_t)BS + threadIdx.x; item < w.total; item += (int64_t)gridDim.x * BS)
        evalres_item(L, w, item, Fs, Gs, BS);
}

// Symmetric pairs of shape (N, N), (N, N-1) or (N-1, N): the same lane pairs
// as k_evalres, but the evaluated columns stay in registers (handed across by
// shuffles) and res_chain solves in registers.  A warp with a lane whose
// subproblem needs the general solver is appended to `redo` and written by
// k_evalres_redo instead (whole warps, since lane pairs share evaluations).
// blocks of 256 per SM the register allocation must allow: three (80 registers,
// a few spills to L1)
// measured fastest at N = 20 (12.0 against 12.5 ms with 128 registers on the
// 4096-pair degree-20 batch); larger N need more registers than that
constexpr int reg_min_blocks(int N) { return N <= 20 ? 3 : N <= 27 ? 2 : 1; }

template <int N>
__global__ void __launch_bounds__(256, reg_min_blocks(N)) k_evalres_reg(ResLaunch L, WorkList w, unsigned long long *redo_n,
                                                     int64_t *redo) {
    for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < w.total;
         item += (int64_t)gridDim.x * blockDim.x) {
        const int bi = wl_find(w.start, w.n, item);
        const int q = w.pairs[bi];
        const int64_t local = item - w.start[bi];
        const PairPlan &P = L.plan[q];
        const int per = P.tiles * 32;
        const int i = (int)(local / per);
        const int r = (int)(local % per);
        const int lane = r & 31;
        const int ii = (r >> 5) * 16 + (lane & 15);
        const bool glane = lane >= 16;
        const int j = ii == 0 ? (glane ? -1 : 0) : (glane ? 2 * ii : 2 * ii - 1);
        const ModP M = L.mods[prime_of(P, L.pmap, i)];
        // even and odd parts at b = ii^2 (an exact integer below p) by Shoup steps on
        // the stored c R^2 residues, so the parts come out as R^2 E and R^2 O
        const uint32_t b = (uint32_t)ii * (uint32_t)ii;
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
                    // R E = redc(R^2 E); R ii O = redc(R^2 O ii) (R^2 O < 3p, so
                    // both inputs stay below p 2^32)
                    const uint32_t ev = mp_redc(e[t], 0u, M.p, M.pinv);
                    const uint32_t io = mp_mul(o[t], (uint32_t)ii, M);
                    const uint32_t plus = mp_add(ev, io, M.p), minus = mp_sub(ev, io, M.p);
                    own[r0 + t] = glane ? minus : plus;
                    oth[r0 + t] = glane ? plus : minus;
                }
            }
        }
        uint32_t F[N + 1], G[N + 1];
#pragma unroll
        for (int k = 0; k <= N; ++k) {
            const uint32_t got = __shfl_xor_sync(0xffffffffu, oth[k], 16);
            F[k] = glane ? got : own[k];
            G[k] = glane ? own[k] : got;
        }
        bool ok;
        const uint32_t v = res_chain<N>(F, G, P.m, P.n, M, ok);
        const bool valid = j >= 0 && j < P.Pe;
        if (__ballot_sync(0xffffffffu, valid && !ok)) {
            if (lane == 0) redo[atomicAdd(redo_n, 1ull)] = item;
        } else if (valid) {
            L.val[P.val_off + (int64_t)i * P.Pe + j] = v;
        }
    }
}

// The warps listed by k_evalres_reg, solved on shared-memory columns.
__global__ void k_evalres_redo(ResLaunch L, WorkList w, int SF, const unsigned long long *redo_n,
                               const int64_t *redo) {
    extern __shared__ uint32_t smem[];
    const int BS = blockDim.x;
    uint32_t *Fs = smem + threadIdx.x;
    uint32_t *Gs = smem + SF * BS + threadIdx.x;
    const int64_t nw = (int64_t)*redo_n;
    const int lane = threadIdx.x & 31;
    for (int64_t e = (blockIdx.x * (int64_t)BS + threadIdx.x) >> 5; e < nw; e += ((int64_t)gridDim.x * BS) >> 5)
        evalres_item(L, w, redo[e] + lane, Fs, Gs, BS);
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
