// Host helpers of the bivariate gcd by Kronecker substitution and of the
// Teissier resultant (internal): the map-back degree, the choice of the
// candidate z^t G / z^v whose map-back is an exact factorisation, the shifts
// y -> y + s of the inputs and back, the partial derivatives of an int64 curve
// and the conversion of big-integer cofactors to two's-complement words.  Host
// code only; kept apart from the CUDA file so the tests can build it on the CPU.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/gbres.h"
#include "gbr_bigint.h"

namespace gbr {
namespace kron {

// x-degree of the map-back of z^off times a Kronecker image with D columns (-1
// for zero); every non-zero coefficient of g sits at an exponent k with k + off >= 0
inline int back_degx(const gbr_bigpoly &g, int D, int off) {
    int dx = -1;
    for (int k = 0; k <= g.deg; ++k)
        if (g.sign[k]) dx = std::max(dx, (k + off) % D);
    return dx;
}

// lowest exponent with a non-zero coefficient (-1 for zero)
inline int valuation(const gbr_bigpoly &g) {
    for (int k = 0; k <= g.deg; ++k)
        if (g.sign[k]) return k;
    return -1;
}

// The shift sh (candidate z^(v - sh) G / z^v with cofactors z^sh phi(a) / G and
// z^sh phi(b) / G, v the multiplicity of z in G) that maps back to a factorisation
// in Z[x][y], trying sh = 0, 1, ..., v (the largest candidate first); 0 for G = 0;
// -1 when none does (a spurious common factor of the images: D must grow).
inline int kron_shift(const gbr_bigpoly &g, const gbr_bigpoly &ga, const gbr_bigpoly &gb, int D) {
    if (g.deg < 0) return 0;
    const int v = valuation(g);
    for (int sh = 0; sh <= v; ++sh) {
        const int dh = back_degx(g, D, -sh), da = back_degx(ga, D, sh), db = back_degx(gb, D, sh);
        if (dh + std::max(da, 0) < D && dh + std::max(db, 0) < D) return sh;
    }
    return -1;
}

// in[j][i] (dx + 1 columns, dy + 1 rows) -> in(x, y + s), column by column (Taylor
// shift in y by repeated synthetic division); false on int64 overflow
inline bool shift_y_i64(const int64_t *in, int dx, int dy, int s, std::vector<int64_t> &out) {
    out.assign(in, in + (size_t)(dx + 1) * (dy + 1));
    for (int i = 0; i <= dx; ++i)
        for (int k = 0; k < dy; ++k)
            for (int j = dy - 1; j >= k; --j) {
                int64_t t;
                if (__builtin_mul_overflow(out[(size_t)(j + 1) * (dx + 1) + i], (int64_t)s, &t) ||
                    __builtin_add_overflow(out[(size_t)j * (dx + 1) + i], t, &out[(size_t)j * (dx + 1) + i]))
                    return false;
            }
    return true;
}

// g(x, y) -> g(x, y - s) in exact big integers, g[j (dx + 1) + i] the coefficient
// of x^i y^j (the inverse of shift_y_i64 with the same s)
inline void unshift_y_big(std::vector<bn::Big> &g, int dx, int dy, int s) {
    const bn::Big ms = bn::from_i64(-(int64_t)s);
    for (int i = 0; i <= dx; ++i)
        for (int k = 0; k < dy; ++k)
            for (int j = dy - 1; j >= k; --j) {
                bn::Big &cj = g[(size_t)j * (dx + 1) + i];
                cj = bn::add(cj, bn::mul(g[(size_t)(j + 1) * (dx + 1) + i], ms));
            }
}

// derivative of an int64 curve in x (wx = true) or y, into `buf`, with `out`
// describing it (dense extents one lower in the variable, at least 0); false on
// int64 overflow
inline bool derive(const gbr_bipoly &f, bool wx, std::vector<int64_t> &buf, gbr_bipoly &out) {
    const int dx = f.deg_x, dy = f.deg_y;
    const int ox = wx ? std::max(dx - 1, 0) : dx, oy = wx ? dy : std::max(dy - 1, 0);
    buf.assign((size_t)(ox + 1) * (oy + 1), 0);
    const int64_t *cf = (const int64_t *)f.coef;
    for (int j = 0; j <= oy; ++j)
        for (int i = 0; i <= ox; ++i) {
            const int si = wx ? i + 1 : i, sj = wx ? j : j + 1;
            if (si > dx || sj > dy) continue;
            const int64_t v = cf[(size_t)sj * (dx + 1) + si], k = wx ? si : sj;
            int64_t r;
            if (__builtin_mul_overflow(v, k, &r)) return false;
            buf[(size_t)j * (ox + 1) + i] = r;
        }
    out.deg_x = ox;
    out.deg_y = oy;
    out.words = 1;
    out.coef = buf.data();
    return true;
}

// a sign-magnitude big bivariate polynomial as two's-complement 64-bit words
// (enough words for the magnitude and a sign bit), into `buf`, with `out`
// describing it; the zero polynomial becomes one coefficient 0; false when more
// than GBR_MAX_WORDS words would be needed
inline bool to_words(const gbr_bigbipoly &x, std::vector<uint64_t> &buf, gbr_bipoly &out) {
    if (x.deg_y < 0) {
        buf.assign(1, 0);
        out.deg_x = out.deg_y = 0;
        out.words = 1;
        out.coef = buf.data();
        return true;
    }
    const int L = x.c.limbs, W = (L * 32 + 1 + 63) / 64;
    if (W > GBR_MAX_WORDS) return false;
    const int nco = (x.deg_x + 1) * (x.deg_y + 1);
    buf.assign((size_t)nco * W, 0);
    for (int t = 0; t < nco; ++t) {
        uint64_t *w = buf.data() + (size_t)t * W;
        for (int l = 0; l < L; ++l) w[l / 2] |= (uint64_t)x.c.mag[(size_t)t * L + l] << (32 * (l % 2));
        if (x.c.sign[t] < 0) {   // negate in two's complement
            uint64_t carry = 1;
            for (int k = 0; k < W; ++k) {
                w[k] = ~w[k] + carry;
                carry = (carry && w[k] == 0) ? 1 : 0;
            }
        }
    }
    out.deg_x = x.deg_x;
    out.deg_y = x.deg_y;
    out.words = W;
    out.coef = buf.data();
    return true;
}

}  // namespace kron
}  // namespace gbr
