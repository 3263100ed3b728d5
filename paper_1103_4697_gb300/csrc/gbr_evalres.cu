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

__global__ void k_evalres(ResLaunch L, WorkList w, int SF, int SG) {
    extern __shared__ uint32_t smem[];
    const int BS = blockDim.x;
    uint32_t *Fs = smem + threadIdx.x;
    uint32_t *Gs = smem + SF * BS + threadIdx.x;
    for (int64_t item = blockIdx.x * (int64_t)BS + threadIdx.x; item < w.total; item += (int64_t)gridDim.x * BS) {
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
            if (j >= 0 && j < P.P)
                L.val[P.val_off + (int64_t)i * P.Pe + j] = res_formal(Fs, P.m, Gs, P.n, BS, M);
            __syncwarp();
            continue;
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
}


cudaError_t launch_evalres(const ResLaunch &L, const WorkList &w, int SF, int SG, int block, cudaStream_t s) {
    if (w.total <= 0) return cudaSuccess;
    size_t smem = (size_t)(SF + SG) * block * sizeof(uint32_t);
    if (smem > kMaxDynSmem) return cudaErrorInvalidValue;
    int grid = persistent_grid(k_evalres, block, smem, (w.total + block - 1) / block);
    k_evalres<<<grid, block, smem, s>>>(L, w, SF, SG);
    return cudaGetLastError();
}


cudaError_t configure_evalres_kernel() {
    return cudaFuncSetAttribute(k_evalres, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

}  // namespace gbr
