// Host big integers for the square-free factorisation (internal): sign and
// magnitude in little-endian 32-bit limbs.  Only what the lift needs: products,
// exact and Euclidean division (Knuth's long division), gcd, comparison.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace gbr {
namespace bn {

struct Big {
    std::vector<uint32_t> m;   // magnitude, no leading zero limbs; empty = 0
    int s = 0;                 // -1, 0, +1
};

inline void trim(Big &a) {
    while (!a.m.empty() && a.m.back() == 0u) a.m.pop_back();
    if (a.m.empty()) a.s = 0;
    else if (a.s == 0) a.s = 1;
}

inline Big from_limbs(const uint32_t *x, int n, int sign) {
    Big a;
    a.m.assign(x, x + n);
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

inline int cmp_mag(const std::vector<uint32_t> &a, const std::vector<uint32_t> &b) {
    if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
    for (size_t i = a.size(); i-- > 0;)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

inline std::vector<uint32_t> mul_mag(const std::vector<uint32_t> &a, const std::vector<uint32_t> &b) {
    if (a.empty() || b.empty()) return {};
    std::vector<uint32_t> r(a.size() + b.size(), 0u);
    for (size_t i = 0; i < a.size(); ++i) {
        uint64_t carry = 0;
        for (size_t j = 0; j < b.size(); ++j) {
            const uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
            r[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        r[i + b.size()] = (uint32_t)carry;
    }
    while (!r.empty() && r.back() == 0u) r.pop_back();
    return r;
}

inline Big mul(const Big &a, const Big &b) {
    Big r;
    r.m = mul_mag(a.m, b.m);
    r.s = a.s * b.s;
    trim(r);
    return r;
}

// q = a / b, r = a mod b for magnitudes (b non-zero): Knuth's algorithm D with
// 32-bit digits, normalised so that the divisor's top digit has its high bit set
inline void divmod_mag(const std::vector<uint32_t> &a, const std::vector<uint32_t> &b, std::vector<uint32_t> &q,
                       std::vector<uint32_t> &r) {
    q.clear();
    r.clear();
    if (cmp_mag(a, b) < 0) {
        r = a;
        return;
    }
    const size_t n = b.size(), m = a.size() - n;
    if (n == 1) {
        q.assign(a.size(), 0u);
        uint64_t rem = 0;
        for (size_t i = a.size(); i-- > 0;) {
            const uint64_t cur = (rem << 32) | a[i];
            q[i] = (uint32_t)(cur / b[0]);
            rem = cur % b[0];
        }
        while (!q.empty() && q.back() == 0u) q.pop_back();
        if (rem) r = {(uint32_t)rem};
        return;
    }
    int sh = 0;
    while (!(b[n - 1] & (0x80000000u >> sh))) ++sh;
    std::vector<uint32_t> v(n), u(a.size() + 1, 0u);
    for (size_t i = n; i-- > 0;) v[i] = (b[i] << sh) | (sh && i ? b[i - 1] >> (32 - sh) : 0u);
    for (size_t i = a.size(); i-- > 0;) {
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
    while (!q.empty() && q.back() == 0u) q.pop_back();
    r.assign(n, 0u);
    for (size_t i = 0; i < n; ++i) r[i] = (u[i] >> sh) | (sh ? (uint32_t)((uint64_t)u[i + 1] << (32 - sh)) : 0u);
    while (!r.empty() && r.back() == 0u) r.pop_back();
}

// a / b when b divides a exactly; false otherwise (b non-zero)
inline bool divexact(const Big &a, const Big &b, Big &q) {
    std::vector<uint32_t> r;
    divmod_mag(a.m, b.m, q.m, r);
    q.s = a.s * b.s;
    trim(q);
    return r.empty();
}

inline std::vector<uint32_t> gcd_mag(std::vector<uint32_t> a, std::vector<uint32_t> b) {
    std::vector<uint32_t> q, r;
    while (!b.empty()) {
        divmod_mag(a, b, q, r);
        a.swap(b);
        b.swap(r);
    }
    return a;
}

inline double log2_mag(const std::vector<uint32_t> &a) {
    if (a.empty()) return -1e300;
    const size_t t = a.size() - 1;
    double v = (double)a[t];
    if (t >= 1) v += (double)a[t - 1] * 0x1p-32;
    if (t >= 2) v += 0x1p-64 * 2.0;   // the truncated tail, rounded up
    return std::log2(v) + 32.0 * (double)t;
}

}  // namespace bn
}  // namespace gbr
