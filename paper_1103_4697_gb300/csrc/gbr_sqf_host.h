// Host helpers of the square-free factorisation (internal): flat factor storage,
// coefficient norms rounded up, and primitive parts of lifted factors.  Host code
// only; kept apart from the CUDA file so the tests can build it on the CPU.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "gbr_bigint.h"

namespace gbr {
namespace sqfh {

// one factor r_i: deg + 1 coefficients of L limbs each, and their signs
struct FlatPoly {
    int deg = -1, L = 1;
    std::vector<uint32_t> mag;
    std::vector<int8_t> sign;
};

// log2 of the 1-, 2- and max-norms of `count` coefficients, rounded up; get(t,
// x, n) gives coefficient t's trimmed magnitude (n = 0 for zero).  Each
// magnitude is bounded from its top two limbs relative to the longest one, so
// the sums need no logarithm per coefficient; -1e300 for the zero polynomial.
struct Norms {
    double l1 = -1e300, l2 = -1e300, linf = -1e300;
};
template <class Get>
Norms log2_norms(int count, Get get) {
    size_t ref = 0;
    for (int t = 0; t < count; ++t) {
        const uint32_t *x;
        size_t n;
        get(t, x, n);
        ref = std::max(ref, n);
    }
    Norms r;
    if (!ref) return r;
    double s1 = 0.0, s2 = 0.0, mx = 0.0;
    for (int t = 0; t < count; ++t) {
        const uint32_t *x;
        size_t n;
        get(t, x, n);
        const double v = bn::scaled_mag(x, n, ref);
        s1 += v;
        s2 += v * v;
        mx = std::max(mx, v);
    }
    const double e = 32.0 * (double)(ref - 1), pad = 1e-9 + 1e-12 * count;
    r.l1 = std::log2(s1) + e + pad;
    r.l2 = 0.5 * std::log2(s2) + e + pad;
    r.linf = std::log2(mx) + e + pad;
    return r;
}

// primitive part with a positive leading coefficient of the lifted factor whose
// d + 1 coefficients (LL limbs each) start at x, signs at sg; false when the
// lift cannot be a multiple of a factor of R (zero leading coefficient).  The
// content g starts as the leading coefficient; every coefficient is divided by
// the current g and a non-zero remainder r replaces g by gcd(g, r) (= gcd(g, c)),
// after which the coefficients already divided are divided again.
inline bool primitive_part(const uint32_t *x, const int8_t *sg, int d, int LL, FlatPoly &f, bn::Scratch &S) {
    if (sg[d] == 0) return false;
    bn::Limbs &g = S.g;
    g.assign(x + (size_t)d * LL, x + (size_t)d * LL + bn::top(x + (size_t)d * LL, LL));
    const int flip = sg[d] < 0 ? -1 : 1;
    f.deg = d;
    f.sign.resize(d + 1);
    f.mag.assign((size_t)(d + 1) * LL, 0u);
    int redo_to = -1;   // coefficients d .. redo_to were divided by an older g
    for (int t = d; t >= 0; --t) {
        f.sign[t] = (int8_t)(sg[t] * flip);
        if (!sg[t] || (g.size() == 1 && g[0] == 1u)) continue;
        const uint32_t *c = x + (size_t)t * LL;
        bn::divmod_mag(c, bn::top(c, LL), g.data(), g.size(), S.q, S.r, S);
        if (!S.r.empty()) {
            S.x = S.r;
            bn::gcd_into(g, S.x.data(), S.x.size(), S);
            redo_to = t;
            continue;
        }
        std::fill(f.mag.begin() + (size_t)t * LL, f.mag.begin() + (size_t)(t + 1) * LL, 0u);
        std::copy(S.q.begin(), S.q.end(), f.mag.begin() + (size_t)t * LL);
    }
    const bool unit = g.size() == 1 && g[0] == 1u;
    int L = 1;
    for (int t = d; t >= 0; --t) {
        if (!sg[t]) continue;
        const uint32_t *c = x + (size_t)t * LL;
        uint32_t *o = f.mag.data() + (size_t)t * LL;
        if (unit) {
            const size_t nl = bn::top(c, LL);
            std::copy(c, c + nl, o);
            std::fill(o + nl, o + LL, 0u);
            L = std::max(L, (int)nl);
            continue;
        }
        if (redo_to >= 0 && t >= redo_to) {
            bn::divmod_mag(c, bn::top(c, LL), g.data(), g.size(), S.q, S.r, S);
            if (!S.r.empty()) return false;
            std::fill(o, o + LL, 0u);
            std::copy(S.q.begin(), S.q.end(), o);
        }
        L = std::max(L, (int)bn::top(o, LL));
    }
    if (L < LL) {   // compact to L limbs per coefficient
        for (int t = 1; t <= d; ++t)
            std::copy(f.mag.begin() + (size_t)t * LL, f.mag.begin() + (size_t)t * LL + L, f.mag.begin() + (size_t)t * L);
        f.mag.resize((size_t)(d + 1) * L);
    }
    f.L = L;
    return true;
}

inline bn::Big lead(const FlatPoly &f) {
    return bn::from_limbs(f.mag.data() + (size_t)f.deg * f.L, f.L, f.sign[f.deg]);
}

}  // namespace sqfh
}  // namespace gbr
