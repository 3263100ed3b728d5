// gcd in Z[x][y] with cofactors, and the Teissier resultant Q (Section 2.1):
// h = gcd(f_x, f_y), f_x* = f_x / h, f_y* = f_y / h, Q = res(f_x*, f_y*, y).
//
// Method: Kronecker substitution onto the device gcd path.  With D larger than
// every x-degree involved, phi(x^i y^j) = z^(i + j D) maps a product whose
// x-degrees add up to less than D onto the product of the images.  The gcd path
// returns, with its exact certificate, G = gcd(phi(A), phi(B)) in Z[z] and the
// cofactors phi(A) / G, phi(B) / G; mapped back (exponent k -> (k mod D, k div D))
// they give H', A', B'.  When deg_x H' + deg_x A' < D and deg_x H' + deg_x B' < D
// the identities A = H' A' and B = H' B' hold in Z[x][y] (phi is injective on
// x-degrees below D), so H' is a common divisor; the true gcd H maps onto a
// divisor of G = phi(H'), and H' | H, so H' = H up to a unit, fixed by the
// positive leading coefficient both carry.
// Powers of z: the images of two polynomials without constant terms share a
// power of z that need not come from a common factor (x + y and x - y give
// z + z^D and z - z^D).  With v the multiplicity of z in G, phi(H) = z^w H1 with
// w <= v and H1 dividing G / z^v; the candidates z^t G / z^v are tried for
// t = v, v - 1, ..., 0 (the cofactors multiplied by z^(v - t)) and the first that
// maps back exactly is taken: the largest such t is at least w, so phi(H) divides
// that candidate and it is H.  When no t passes (G holds another common factor of
// the images that is not an image of one), the job runs again with D doubled.
#include <cstring>
#include <vector>

#include "gbr_core.h"

using namespace gbr;

namespace {

// x-degree of the map-back of z^off times a Kronecker image with D columns (-1
// for zero); every non-zero coefficient of g sits at an exponent k with k + off >= 0
int back_degx(const gbr_bigpoly &g, int D, int off) {
    int dx = -1;
    for (int k = 0; k <= g.deg; ++k)
        if (g.sign[k]) dx = std::max(dx, (k + off) % D);
    return dx;
}

// lowest exponent with a non-zero coefficient (-1 for zero)
int valuation(const gbr_bigpoly &g) {
    for (int k = 0; k <= g.deg; ++k)
        if (g.sign[k]) return k;
    return -1;
}

// the map-back of z^off g into [deg_y][deg_x] layout
bool map_back(const gbr_bigpoly &g, int D, int off, gbr_bigbipoly &out) {
    out.deg_x = out.deg_y = -1;
    out.c = gbr_bigpoly{-1, 0, nullptr, nullptr};
    if (g.deg < 0) return true;
    const int dx = back_degx(g, D, off), dy = (g.deg + off) / D;
    out.deg_x = dx;
    out.deg_y = dy;
    out.c.deg = (dx + 1) * (dy + 1) - 1;
    out.c.limbs = g.limbs;
    if (!gbr_alloc_results(&out.c, 1)) return false;
    std::memset(out.c.mag, 0, (size_t)(out.c.deg + 1) * out.c.limbs * 4);
    std::memset(out.c.sign, 0, (size_t)out.c.deg + 1);
    for (int k = 0; k <= g.deg; ++k) {
        if (!g.sign[k]) continue;
        const int i = (k + off) % D, j = (k + off) / D, t = j * (dx + 1) + i;
        std::memcpy(out.c.mag + (size_t)t * out.c.limbs, g.mag + (size_t)k * g.limbs, (size_t)g.limbs * 4);
        out.c.sign[t] = g.sign[k];
    }
    return true;
}

void clear(gbr_bigbipoly &x) {
    x.deg_x = x.deg_y = -1;
    x.c = gbr_bigpoly{-1, 0, nullptr, nullptr};
}

}  // namespace

static int gcd2_locked(gbr_ctx *c, int n, const gbr_bipoly *a, const gbr_bipoly *b, gbr_bigbipoly *h,
                       gbr_bigbipoly *ah, gbr_bigbipoly *bh) {
    for (int i = 0; i < n; ++i) {
        for (const gbr_bipoly *x : {&a[i], &b[i]})
            if (!x->coef || x->deg_x < 0 || x->deg_y < 0 || x->words != 1)
                return c->fail(GBR_EINVAL, "bivariate gcd inputs must be int64 bipolys (words = 1)");
        clear(h[i]);
        clear(ah[i]);
        clear(bh[i]);
    }
    std::vector<int> D(n), pend(n);
    for (int i = 0; i < n; ++i) {
        D[i] = std::max(a[i].deg_x, b[i].deg_x) + 1;
        pend[i] = i;
    }
    while (!pend.empty()) {
        const int m = (int)pend.size();
        std::vector<std::vector<int64_t>> za(m), zb(m);
        std::vector<gbr_upoly> up(m), uq(m);
        for (int t = 0; t < m; ++t) {
            const int i = pend[t];
            for (int w = 0; w < 2; ++w) {
                const gbr_bipoly &x = w ? b[i] : a[i];
                std::vector<int64_t> &z = w ? zb[t] : za[t];
                const int64_t deg = (int64_t)x.deg_y * D[i] + x.deg_x;
                if (deg > GBR_MAX_UDEG)
                    return c->fail(GBR_ELIMIT, "bivariate gcd: Kronecker image above GBR_MAX_UDEG");
                z.assign((size_t)deg + 1, 0);
                const int64_t *cf = (const int64_t *)x.coef;
                for (int j = 0; j <= x.deg_y; ++j)
                    for (int k = 0; k <= x.deg_x; ++k) z[(size_t)j * D[i] + k] = cf[(size_t)j * (x.deg_x + 1) + k];
                gbr_upoly &u = w ? uq[t] : up[t];
                u.deg = (int32_t)deg;
                u.words = 1;
                u.coef = z.data();
            }
        }
        std::vector<gbr_bigpoly> g(m), ga(m), gb(m);
        int st = gbr_gcd_cof_locked(c, m, up.data(), uq.data(), g.data(), ga.data(), gb.data());
        if (st) return st;
        std::vector<int> retry;
        int rc = GBR_OK;
        for (int t = 0; t < m && rc == GBR_OK; ++t) {
            const int i = pend[t];
            int shift = -1;   // the candidate z^(v - shift) G / z^v that maps back exactly
            if (g[t].deg < 0) {
                shift = 0;
            } else {
                const int v = valuation(g[t]);
                for (int sh = 0; sh <= v && shift < 0; ++sh) {
                    const int dh = back_degx(g[t], D[i], -sh), da = back_degx(ga[t], D[i], sh),
                              db = back_degx(gb[t], D[i], sh);
                    if (dh + std::max(da, 0) < D[i] && dh + std::max(db, 0) < D[i]) shift = sh;
                }
            }
            if (shift < 0) {
                retry.push_back(i);
            } else if (!map_back(g[t], D[i], -shift, h[i]) || !map_back(ga[t], D[i], shift, ah[i]) ||
                       !map_back(gb[t], D[i], shift, bh[i])) {
                rc = c->fail(GBR_ENOMEM, "host result allocation");
            }
        }
        for (int t = 0; t < m; ++t) {
            gbr_free_result(c, &g[t]);
            gbr_free_result(c, &ga[t]);
            gbr_free_result(c, &gb[t]);
        }
        if (rc) return rc;
        for (int i : retry) D[i] *= 2;
        pend.swap(retry);
    }
    return GBR_OK;
}

extern "C" int gbr_gcd2_batch(gbr_ctx *c, int n, const gbr_bipoly *a, const gbr_bipoly *b, gbr_bigbipoly *h,
                              gbr_bigbipoly *a_over_h, gbr_bigbipoly *b_over_h) {
    if (!c || n < 0 || (n && (!a || !b || !h || !a_over_h || !b_over_h))) return GBR_EINVAL;
    if (n == 0) return GBR_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    int st;
    try {
        st = gcd2_locked(c, n, a, b, h, a_over_h, b_over_h);
    } catch (std::bad_alloc &) {
        st = c->fail(GBR_ENOMEM, "host allocation");
    }
    if (st)
        for (int i = 0; i < n; ++i) {
            gbr_free_bigbipoly(c, &h[i]);
            gbr_free_bigbipoly(c, &a_over_h[i]);
            gbr_free_bigbipoly(c, &b_over_h[i]);
        }
    return st;
}

extern "C" void gbr_free_bigbipoly(gbr_ctx *c, gbr_bigbipoly *x) {
    if (!x) return;
    gbr_free_result(c, &x->c);
    x->deg_x = x->deg_y = -1;
}

// ------------------------------------------------------------------ Teissier resultant

namespace {

// derivative of an int64 bipoly in x (wx = true) or y, into `buf`; false on overflow
bool derive(const gbr_bipoly &f, bool wx, std::vector<int64_t> &buf, gbr_bipoly &out) {
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

// a sign-magnitude bigbipoly as an array of two's-complement 64-bit words
bool to_words(const gbr_bigbipoly &x, std::vector<uint64_t> &buf, gbr_bipoly &out) {
    if (x.deg_y < 0) {   // zero: one coefficient 0
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

}  // namespace

extern "C" int gbr_teissier_res_batch(gbr_ctx *c, int n, const gbr_bipoly *f, gbr_bigpoly *q) {
    if (!c || n < 0 || (n && (!f || !q))) return GBR_EINVAL;
    for (int i = 0; i < n; ++i) q[i] = gbr_bigpoly{-1, 0, nullptr, nullptr};
    if (n == 0) return GBR_OK;
    std::vector<std::vector<int64_t>> bx(n), by(n);
    std::vector<gbr_bipoly> fx(n), fy(n);
    for (int i = 0; i < n; ++i) {
        if (!f[i].coef || f[i].deg_x < 0 || f[i].deg_y < 0 || f[i].words != 1) return GBR_EINVAL;
        if (!derive(f[i], true, bx[i], fx[i]) || !derive(f[i], false, by[i], fy[i])) return GBR_ELIMIT;
    }
    std::vector<gbr_bigbipoly> h(n), fxs(n), fys(n);
    int st = gbr_gcd2_batch(c, n, fx.data(), fy.data(), h.data(), fxs.data(), fys.data());
    if (st) return st;
    std::vector<std::vector<uint64_t>> wa(n), wb(n);
    std::vector<gbr_bipoly> A(n), B(n);
    for (int i = 0; i < n && !st; ++i)
        if (!to_words(fxs[i], wa[i], A[i]) || !to_words(fys[i], wb[i], B[i])) st = GBR_ELIMIT;
    if (!st) st = gbr_resultant_batch(c, n, A.data(), B.data(), 1, q);
    for (int i = 0; i < n; ++i) {
        gbr_free_bigbipoly(c, &h[i]);
        gbr_free_bigbipoly(c, &fxs[i]);
        gbr_free_bigbipoly(c, &fys[i]);
    }
    return st;
}
