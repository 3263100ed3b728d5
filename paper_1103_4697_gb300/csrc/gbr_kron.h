// Host helpers of the bivariate gcd by Kronecker substitution (internal): the
// map-back degree and the choice of the candidate z^t G / z^v whose map-back is
// an exact factorisation.  Host code only; kept apart from the CUDA file so the
// tests can build it on the CPU.
#pragma once
#include <algorithm>

#include "../../include/gbres.h"

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

}  // namespace kron
}  // namespace gbr
