// The per-(prime, point) resultant over F_p (step A3 of the path): the general
// formal-degree recursion res_formal on strided columns and the register form
// res_chain<N> for the common shapes.  Host and device (GBR_HD): the evaluation
// kernels use them on the GPU, and the tests run the same code on the CPU.
#pragma once
#include <stdint.h>

#include "gbr_modarith.cuh"

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

// The register form as a fraction: the resultant is num / den (den != 0; den = 1
// in Montgomery form when num = 0), so that the caller can batch the inversions.
template <int N>
GBR_HD uint32_t res_chain_frac(const uint32_t (&F)[N + 1], const uint32_t (&G)[N + 1], int m, int n, const ModP &M,
                               bool &ok, uint32_t &den_out) {
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
    den_out = M.r1;
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
    den_out = mp_mul(den, Dq, M);
    return acc;
}

template <int N>
GBR_HD uint32_t res_chain(const uint32_t (&F)[N + 1], const uint32_t (&G)[N + 1], int m, int n, const ModP &M,
                          bool &ok) {
    uint32_t den;
    const uint32_t num = res_chain_frac<N>(F, G, m, n, M, ok, den);
    return mp_mul(num, mp_inv(den, M), M);
}

}  // namespace gbr
