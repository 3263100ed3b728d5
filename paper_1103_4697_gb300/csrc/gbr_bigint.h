// Host big integers for the square-free factorisation (internal): sign and
// magnitude in little-endian 32-bit limbs.  Only what the lift needs: products,
// exact and Euclidean division (Knuth's long division), gcd, comparison.  The
// division and gcd work on limb slices with caller-provided scratch vectors, so
// a loop over many coefficients allocates nothing once the scratch has grown.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace gbr {
namespace bn {

using Limbs = std::vector<uint32_t>;

struct Big {
    Limbs m;     // magnitude, no leading zero limbs; empty = 0
    int s = 0;   // -1, 0, +1
};

// reusable buffers of one thread
struct Scratch {
    Limbs u, v, q, r, a, b, g, x;
};

inline size_t top(const uint32_t *x, size_t n) {
    while (n && x[n - 1] == 0u) --n;
    return n;
}

inline void trim(Big &a) {
    a.m.resize(top(a.m.data(), a.m.size()));
    if (a.m.empty()) a.s = 0;
    else if (a.s == 0) a.s = 1;
}

inline Big from_limbs(const uint32_t *x, int n, int sign) {
    Big a;
    a.m.assign(x, x + top(x, (size_t)n));
    a.s = sign < 0 ? -1 : 1;
    trim(a);
    return a;
}

inline Big from_u64(uint64_t v, int sign = 1) {
    Big a;
    a.m = {(uint32_t)v, (uint32_t)(v >> 32)};
    a.s = sign;
    trim(a);
    return a;
}

inline int cmp_mag(const uint32_t *a, size_t na, const uint32_t *b, size_t nb) {
    if (na != nb) return na < nb ? -1 : 1;
    for (size_t i = na; i-- > 0;)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

inline Limbs mul_mag(const Limbs &a, const Limbs &b) {
    if (a.empty() || b.empty()) return {};
    Limbs r(a.size() + b.size(), 0u);
    for (size_t i = 0; i < a.size(); ++i) {
        uint64_t carry = 0;
        for (size_t j = 0; j < b.size(); ++j) {
            const uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
            r[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        r[i + b.size()] = (uint32_t)carry;
    }
    r.resize(top(r.data(), r.size()));
    return r;
}

// |a| + |b| and |a| - |b| (|a| >= |b|) for trimmed magnitudes
inline Limbs add_mag(const Limbs &a, const Limbs &b) {
    const Limbs &x = a.size() >= b.size() ? a : b, &y = a.size() >= b.size() ? b : a;
    Limbs r(x.size() + 1, 0u);
    uint64_t carry = 0;
    for (size_t i = 0; i < x.size(); ++i) {
        const uint64_t t = (uint64_t)x[i] + (i < y.size() ? y[i] : 0u) + carry;
        r[i] = (uint32_t)t;
        carry = t >> 32;
    }
    r[x.size()] = (uint32_t)carry;
    r.resize(top(r.data(), r.size()));
    return r;
}

inline Limbs sub_mag(const Limbs &a, const Limbs &b) {
    Limbs r(a.size(), 0u);
    int64_t borrow = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        const int64_t t = (int64_t)a[i] - (i < b.size() ? (int64_t)b[i] : 0) + borrow;
        r[i] = (uint32_t)t;
        borrow = t >> 32;
    }
    r.resize(top(r.data(), r.size()));
    return r;
}

// a + b, signed
inline Big add(const Big &a, const Big &b) {
    if (!b.s) return a;
    if (!a.s) return b;
    Big r;
    if (a.s == b.s) {
        r.m = add_mag(a.m, b.m);
        r.s = a.s;
    } else {
        const int c = cmp_mag(a.m.data(), a.m.size(), b.m.data(), b.m.size());
        if (c == 0) return Big();
        r.m = c > 0 ? sub_mag(a.m, b.m) : sub_mag(b.m, a.m);
        r.s = c > 0 ? a.s : b.s;
    }
    trim(r);
    return r;
}

inline Big from_i64(int64_t v) {
    return from_u64(v < 0 ? 0ull - (uint64_t)v : (uint64_t)v, v < 0 ? -1 : 1);
}

inline Big mul(const Big &a, const Big &b) {
    Big r;
    r.m = mul_mag(a.m, b.m);
    r.s = a.s * b.s;
    trim(r);
    return r;
}

// q = a / b, r = a mod b for trimmed magnitudes (nb > 0): Knuth's algorithm D
// with 32-bit digits, normalised so that the divisor's top digit has its high
// bit set.  q and r must not alias a, b or the scratch's u and v.
inline void divmod_mag(const uint32_t *a, size_t na, const uint32_t *b, size_t n, Limbs &q, Limbs &r, Scratch &S) {
    q.clear();
    r.clear();
    if (cmp_mag(a, na, b, n) < 0) {
        r.assign(a, a + na);
        return;
    }
    if (na <= 4) {   // both below 2^128: one double-word division, no normalisation
        unsigned __int128 A = 0, B = 0;
        for (size_t i = na; i-- > 0;) A = (A << 32) | a[i];
        for (size_t i = n; i-- > 0;) B = (B << 32) | b[i];
        const unsigned __int128 Q = A / B, R = A - Q * B;
        for (unsigned __int128 t = Q; t; t >>= 32) q.push_back((uint32_t)t);
        for (unsigned __int128 t = R; t; t >>= 32) r.push_back((uint32_t)t);
        return;
    }
    const size_t m = na - n;
    if (n == 1) {
        q.assign(na, 0u);
        uint64_t rem = 0;
        for (size_t i = na; i-- > 0;) {
            const uint64_t cur = (rem << 32) | a[i];
            q[i] = (uint32_t)(cur / b[0]);
            rem = cur % b[0];
        }
        q.resize(top(q.data(), q.size()));
        if (rem) r.assign(1, (uint32_t)rem);
        return;
    }
    int sh = 0;
    while (!(b[n - 1] & (0x80000000u >> sh))) ++sh;
    Limbs &v = S.v, &u = S.u;
    v.assign(n, 0u);
    u.assign(na + 1, 0u);
    for (size_t i = n; i-- > 0;) v[i] = (b[i] << sh) | (sh && i ? b[i - 1] >> (32 - sh) : 0u);
    for (size_t i = na; i-- > 0;) {
        u[i + 1] |= sh ? a[i] >> (32 - sh) : 0u;
        u[i] = a[i] << sh;
    }
    q.assign(m + 1, 0u);
    for (size_t j = m + 1; j-- > 0;) {
        const uint64_t num = ((uint64_t)u[j + n] << 32) | u[j + n - 1];
        uint64_t qh = num / v[n - 1], rh = num % v[n - 1];
        if (qh > 0xFFFFFFFFull) {   // the top remainder digit equals v's: clamp to b - 1
            qh = 0xFFFFFFFFull;
            rh = num - qh * v[n - 1];
        }
        while (rh <= 0xFFFFFFFFull && qh * v[n - 2] > ((rh << 32) | u[j + n - 2])) {
            --qh;
            rh += v[n - 1];
        }
        int64_t borrow = 0;
        uint64_t carry = 0;
        for (size_t i = 0; i < n; ++i) {
            const uint64_t p = qh * v[i] + carry;
            carry = p >> 32;
            const int64_t t = (int64_t)u[i + j] - (int64_t)(uint32_t)p + borrow;
            u[i + j] = (uint32_t)t;
            borrow = t >> 32;
        }
        const int64_t t = (int64_t)u[j + n] - (int64_t)carry + borrow;
        u[j + n] = (uint32_t)t;
        if (t < 0) {   // added back: the estimate was one too large
            --qh;
            uint64_t c = 0;
            for (size_t i = 0; i < n; ++i) {
                const uint64_t s = (uint64_t)u[i + j] + v[i] + c;
                u[i + j] = (uint32_t)s;
                c = s >> 32;
            }
            u[j + n] += (uint32_t)c;
        }
        q[j] = (uint32_t)qh;
    }
    q.resize(top(q.data(), q.size()));
    r.assign(n, 0u);
    for (size_t i = 0; i < n; ++i) r[i] = (u[i] >> sh) | (sh ? (uint32_t)((uint64_t)u[i + 1] << (32 - sh)) : 0u);
    r.resize(top(r.data(), r.size()));
}

inline void divmod_mag(const Limbs &a, const Limbs &b, Limbs &q, Limbs &r, Scratch &S) {
    divmod_mag(a.data(), a.size(), b.data(), b.size(), q, r, S);
}

// a / b when b (non-zero) divides a exactly; false otherwise
inline bool divexact(const Big &a, const Big &b, Big &q, Scratch &S) {
    divmod_mag(a.m, b.m, q.m, S.r, S);
    q.s = a.s * b.s;
    trim(q);
    return S.r.empty();
}

inline uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// the 62 bits of x starting at bit `shift` (bits beyond the top read as 0)
inline uint64_t bits62(const Limbs &x, size_t shift) {
    const size_t w = shift >> 5, o = shift & 31;
    unsigned __int128 t = 0;
    for (int k = 2; k >= 0; --k) {
        const size_t i = w + (size_t)k;
        t = (t << 32) | (i < x.size() ? x[i] : 0u);
    }
    return (uint64_t)(t >> o) & ((1ull << 62) - 1);
}

// r = A x + B y for the non-negative result of a Lehmer step (A, B of opposite
// signs or zero, |A|, |B| < 2^62)
inline void lin_comb(const Limbs &x, int64_t A, const Limbs &y, int64_t B, Limbs &r) {
    const size_t n = std::max(x.size(), y.size());
    r.assign(n + 2, 0u);
    __int128 acc = 0;
    for (size_t i = 0; i < n + 2; ++i) {
        if (i < x.size()) acc += (__int128)A * x[i];
        if (i < y.size()) acc += (__int128)B * y[i];
        r[i] = (uint32_t)(uint64_t)acc;
        acc >>= 32;   // arithmetic shift: floor division by 2^32
    }
    r.resize(top(r.data(), r.size()));
}

// a <- gcd(a, b) of trimmed magnitudes (b is destroyed) by Lehmer's algorithm
// (Knuth, TAOCP vol. 2, 4.5.2, Algorithm L) on 62-bit leading parts: single-word
// quotient steps collected in a 2x2 cofactor matrix, applied to the full numbers
// once the word quotients become uncertain; word Euclid at the end
inline void gcd_lehmer(Limbs &a, Limbs &b, Scratch &S) {
    if (cmp_mag(a.data(), a.size(), b.data(), b.size()) < 0) a.swap(b);
    while (b.size() > 2) {
        const size_t abits = 32 * a.size() - (size_t)__builtin_clz(a.back());
        const size_t shift = abits - 62;
        int64_t ah = (int64_t)bits62(a, shift), bh = (int64_t)bits62(b, shift);
        int64_t A = 1, B = 0, C = 0, D = 1;
        for (;;) {
            if (bh + C == 0 || bh + D == 0) break;
            const int64_t q = (ah + A) / (bh + C);
            if (q != (ah + B) / (bh + D)) break;
            int64_t t = A - q * C;
            A = C;
            C = t;
            t = B - q * D;
            B = D;
            D = t;
            t = ah - q * bh;
            ah = bh;
            bh = t;
        }
        if (B == 0) {   // no single-word step was certain: one full division
            divmod_mag(a, b, S.q, S.r, S);
            a.swap(b);
            b.swap(S.r);
        } else {
            lin_comb(a, A, b, B, S.q);
            lin_comb(a, C, b, D, S.r);
            a.swap(S.q);
            b.swap(S.r);
        }
    }
    if (b.empty()) return;
    const uint64_t bv = (uint64_t)b[0] | (b.size() > 1 ? (uint64_t)b[1] << 32 : 0ull);
    uint64_t rem = 0;
    for (size_t i = a.size(); i-- > 0;) rem = (uint64_t)((((unsigned __int128)rem << 32) | a[i]) % bv);
    const uint64_t d = gcd64(bv, rem);
    a.assign({(uint32_t)d, (uint32_t)(d >> 32)});
    a.resize(top(a.data(), a.size()));
}

// g <- gcd(g, x) for a trimmed g and the limb slice x (n limbs, maybe with
// leading zeros); g = 0 (empty) is the identity
inline void gcd_into(Limbs &g, const uint32_t *x, size_t n, Scratch &S) {
    n = top(x, n);
    if (!n) return;
    if (g.empty()) {
        g.assign(x, x + n);
        return;
    }
    if (g.size() == 1 && g[0] == 1u) return;
    if (g.size() <= 2) {   // reduce x modulo the small g, then word gcd
        const uint64_t gv = (uint64_t)g[0] | (g.size() > 1 ? (uint64_t)g[1] << 32 : 0ull);
        uint64_t rem = 0;
        for (size_t i = n; i-- > 0;) {
            const unsigned __int128 cur = ((unsigned __int128)rem << 32) | x[i];
            rem = (uint64_t)(cur % gv);
        }
        const uint64_t d = gcd64(gv, rem);
        g.assign({(uint32_t)d, (uint32_t)(d >> 32)});
        g.resize(top(g.data(), g.size()));
        return;
    }
    S.a = g;
    S.b.assign(x, x + n);
    gcd_lehmer(S.a, S.b, S);
    g = S.a;
}

inline double log2_mag(const uint32_t *a, size_t n) {
    n = top(a, n);
    if (!n) return -1e300;
    const size_t t = n - 1;
    double v = (double)a[t];
    if (t >= 1) v += (double)a[t - 1] * 0x1p-32;
    if (t >= 2) v += 0x1p-64 * 2.0;   // the truncated tail, rounded up
    return std::log2(v) + 32.0 * (double)t;
}

inline double log2_mag(const Limbs &a) { return log2_mag(a.data(), a.size()); }

// an upper bound of |x| / 2^(32 (ref - 1)) from the top two limbs of the
// trimmed magnitude x (n limbs, n <= ref), as a double
inline double scaled_mag(const uint32_t *x, size_t n, size_t ref) {
    if (!n) return 0.0;
    double v = (double)x[n - 1] + (n >= 2 ? ((double)x[n - 2] + 1.0) * 0x1p-32 : 0.0);
    return std::ldexp(v * (1.0 + 0x1p-50), 32 * ((int)n - (int)ref));
}

}  // namespace bn
}  // namespace gbr
