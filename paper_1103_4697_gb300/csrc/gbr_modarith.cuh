// Montgomery arithmetic modulo primes below 2^32 / 3 (R = 2^32), integer pipes only.
//
// Every residue on the device path is kept in Montgomery form x~ = x * 2^32 mod p.
// redc(t) = t * 2^-32 mod p for 0 <= t < p * 2^32.  With p < 2^32 / 3 a sum of
// up to three products of residues stays below 3 p^2 < p * 2^32, so one
// reduction serves a fused multiply-subtract of two or three products (the
// elimination steps of the resultant).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GBR_HD __host__ __device__ __forceinline__
#else
#define GBR_HD inline
#endif

struct ModP {
    uint32_t p;      // odd prime, 2^30 < p < 2^32 / 3
    uint32_t pinv;   // -p^-1 mod 2^32
    uint32_t r1;     // 2^32 mod p   (Montgomery form of 1)
    uint32_t r2;     // 2^64 mod p   (to_mont multiplier)
};

GBR_HD uint32_t mp_min(uint32_t a, uint32_t b) { return a < b ? a : b; }

// (hi:lo) * 2^-32 mod p, result in [0, p).  Requires (hi:lo) < p * 2^32.
GBR_HD uint32_t mp_redc(uint32_t lo, uint32_t hi, uint32_t p, uint32_t pinv) {
    uint32_t m = lo * pinv;
#if defined(__CUDA_ARCH__)
    uint32_t r;
    // low word of lo + m*p is zero by construction; only its carry survives
    asm("{\n\t.reg .u32 t;\n\t"
        "mad.lo.cc.u32 t, %1, %2, %3;\n\t"
        "madc.hi.u32 %0, %1, %2, %4;\n\t"
        "}"
        : "=r"(r)
        : "r"(m), "r"(p), "r"(lo), "r"(hi));
    return min(r, r - p);
#else
    uint64_t t = (((uint64_t)hi << 32) | lo) + (uint64_t)m * p;
    uint32_t r = (uint32_t)(t >> 32);
    return r >= p ? r - p : r;
#endif
}

GBR_HD uint32_t mp_mul(uint32_t a, uint32_t b, const ModP &M) {
#if defined(__CUDA_ARCH__)
    return mp_redc(a * b, __umulhi(a, b), M.p, M.pinv);
#else
    uint64_t t = (uint64_t)a * b;
    return mp_redc((uint32_t)t, (uint32_t)(t >> 32), M.p, M.pinv);
#endif
}

// (a*x - b*y) * 2^-32 mod p for residues a, x, b, y in [0, p).
GBR_HD uint32_t mp_mulsub(uint32_t a, uint32_t x, uint32_t b, uint32_t y, const ModP &M) {
    uint32_t nb = M.p - b;   // in (0, p]
#if defined(__CUDA_ARCH__)
    uint32_t lo = a * x, hi = __umulhi(a, x);
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
        "madc.hi.u32 %1, %2, %3, %1;"
        : "+r"(lo), "+r"(hi)
        : "r"(nb), "r"(y));
    return mp_redc(lo, hi, M.p, M.pinv);
#else
    uint64_t t = (uint64_t)a * x + (uint64_t)nb * y;
    return mp_redc((uint32_t)t, (uint32_t)(t >> 32), M.p, M.pinv);
#endif
}

// (a*x + b*y) * 2^-32 mod p for residues in [0, p].
GBR_HD uint32_t mp_fma2(uint32_t a, uint32_t x, uint32_t b, uint32_t y, const ModP &M) {
#if defined(__CUDA_ARCH__)
    uint32_t lo = a * x, hi = __umulhi(a, x);
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
        "madc.hi.u32 %1, %2, %3, %1;"
        : "+r"(lo), "+r"(hi)
        : "r"(b), "r"(y));
    return mp_redc(lo, hi, M.p, M.pinv);
#else
    uint64_t t = (uint64_t)a * x + (uint64_t)b * y;
    return mp_redc((uint32_t)t, (uint32_t)(t >> 32), M.p, M.pinv);
#endif
}

// (a*x + b*y + c*z) * 2^-32 mod p for residues in [0, p] (sum < 3 p^2 < p 2^32).
GBR_HD uint32_t mp_fma3(uint32_t a, uint32_t x, uint32_t b, uint32_t y, uint32_t c, uint32_t z, const ModP &M) {
#if defined(__CUDA_ARCH__)
    uint32_t lo = a * x, hi = __umulhi(a, x);
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
        "madc.hi.u32 %1, %2, %3, %1;\n\t"
        "mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
        "madc.hi.u32 %1, %4, %5, %1;"
        : "+r"(lo), "+r"(hi)
        : "r"(b), "r"(y), "r"(c), "r"(z));
    return mp_redc(lo, hi, M.p, M.pinv);
#else
    uint64_t t = (uint64_t)a * x + (uint64_t)b * y + (uint64_t)c * z;
    return mp_redc((uint32_t)t, (uint32_t)(t >> 32), M.p, M.pinv);
#endif
}

GBR_HD uint32_t mp_add(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t s = a + b;
    return mp_min(s, s - p);
}

GBR_HD uint32_t mp_sub(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t d = a - b;
    return mp_min(d, d + p);
}

GBR_HD uint32_t mp_neg(uint32_t a, uint32_t p) { return a ? p - a : 0; }

// Montgomery form of any 32-bit value v (v need not be reduced).
GBR_HD uint32_t mp_to(uint32_t v, const ModP &M) { return mp_mul(v, M.r2, M); }

GBR_HD uint32_t mp_from(uint32_t x, const ModP &M) { return mp_redc(x, 0u, M.p, M.pinv); }

// x~^e in Montgomery form (square and multiply, e >= 0).
GBR_HD uint32_t mp_pow(uint32_t x, uint32_t e, const ModP &M) {
    uint32_t r = M.r1;
    while (e) {
        if (e & 1u) r = mp_mul(r, x, M);
        e >>= 1;
        if (e) x = mp_mul(x, x, M);
    }
    return r;
}

// Inverse by Fermat's little theorem: x^(p-2); x~ must be non-zero.
GBR_HD uint32_t mp_inv(uint32_t x, const ModP &M) { return mp_pow(x, M.p - 2u, M); }

// Montgomery form of a two's-complement integer held in W little-endian 64-bit words.
GBR_HD uint32_t mp_from_words(const uint64_t *w, int W, const ModP &M) {
    bool neg = (int64_t)w[W - 1] < 0;
    uint32_t acc = 0;
    uint32_t carry = 1;    // for two's-complement negation: ~w + 1
    // process words from the most significant end; negation needs the carry from
    // the least significant end, so negate into a small local copy first
    uint64_t mag[8];
    for (int i = 0; i < W; ++i) {
        uint64_t v = neg ? ~w[i] : w[i];
        if (neg) {
            uint64_t s = v + carry;
            carry = (carry && s == 0) ? 1u : 0u;
            v = s;
        }
        mag[i] = v;
    }
    for (int i = W - 1; i >= 0; --i) {
        uint32_t hi = (uint32_t)(mag[i] >> 32), lo = (uint32_t)mag[i];
        acc = mp_add(mp_mul(acc, M.r2, M), mp_to(hi, M), M.p);
        acc = mp_add(mp_mul(acc, M.r2, M), mp_to(lo, M), M.p);
    }
    return neg ? mp_neg(acc, M.p) : acc;
}
