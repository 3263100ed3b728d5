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
// the images that is not an image of one), the job runs again with D + 1: such a
// factor comes from common zeros (x0, x0^D) of the inputs with x0 a root of unity
// (both inputs vanishing at (-1, 1) put 1 + z into every image with D even), so
// consecutive D leave it behind unless the common zeros cover every residue of D.
// A common zero at (1, 1) defeats every monomial substitution (z - 1 divides
// every image), so after kTriesPerShift values of D the inputs are replaced by
// A(x, y + s), B(x, y + s) for s = 1, 2, 3 (int64 Taylor shifts, moving the common
// zeros), and the results are shifted back by y -> y - s in exact big integers;
// leading coefficients in y and contents are unchanged by the shift.  After the
// last shift the call gives up with GBR_EVERIFY.
#include <cstring>
#include <vector>

#include "gbr_bigint.h"
#include "gbr_core.h"
#include "gbr_kron.h"

using namespace gbr;
using namespace gbr::kron;

namespace {

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

// x <- x(x, y - s) in exact big integers (the inverse of the input shift)
bool unshift_y(gbr_ctx *c, gbr_bigbipoly &x, int s) {
    if (x.deg_y < 1) return true;   // constants in y are unchanged
    const int dx = x.deg_x, dy = x.deg_y, L = x.c.limbs;
    std::vector<bn::Big> g((size_t)(dx + 1) * (dy + 1));
    for (size_t t = 0; t < g.size(); ++t)
        if (x.c.sign[t]) g[t] = bn::from_limbs(x.c.mag + t * L, L, x.c.sign[t]);
    unshift_y_big(g, dx, dy, s);
    size_t nl = 1;
    for (const bn::Big &b : g) nl = std::max(nl, b.m.size());
    gbr_bigbipoly y;
    y.deg_x = dx;
    y.deg_y = dy;
    y.c = gbr_bigpoly{x.c.deg, (int32_t)nl, nullptr, nullptr};
    if (!gbr_alloc_results(&y.c, 1)) return false;
    for (size_t t = 0; t < g.size(); ++t) {
        for (size_t l = 0; l < nl; ++l) y.c.mag[t * nl + l] = l < g[t].m.size() ? g[t].m[l] : 0u;
        y.c.sign[t] = (int8_t)g[t].s;
    }
    gbr_free_result(c, &x.c);
    x = y;
    return true;
}

}  // namespace

static const int kTriesPerShift = 4, kMaxShift = 3;

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
    std::vector<int> D(n), pend(n), D0(n), sh(n, 0), tries(n, 0);
    std::vector<std::vector<int64_t>> sa(n), sb(n);   // shifted inputs (when sh > 0)
    for (int i = 0; i < n; ++i) {
        D[i] = D0[i] = std::max(a[i].deg_x, b[i].deg_x) + 1;
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
                const int64_t *cf = sh[i] ? (w ? sb[i] : sa[i]).data() : (const int64_t *)x.coef;
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
            const int shift = kron_shift(g[t], ga[t], gb[t], D[i]);
            if (shift < 0) {
                retry.push_back(i);
            } else if (!map_back(g[t], D[i], -shift, h[i]) || !map_back(ga[t], D[i], shift, ah[i]) ||
                       !map_back(gb[t], D[i], shift, bh[i]) ||
                       (sh[i] && (!unshift_y(c, h[i], sh[i]) || !unshift_y(c, ah[i], sh[i]) ||
                                  !unshift_y(c, bh[i], sh[i])))) {
                rc = c->fail(GBR_ENOMEM, "host result allocation");
            }
        }
        for (int t = 0; t < m; ++t) {
            gbr_free_result(c, &g[t]);
            gbr_free_result(c, &ga[t]);
            gbr_free_result(c, &gb[t]);
        }
        if (rc) return rc;
        for (int i : retry) {
            ++D[i];
            if (++tries[i] < kTriesPerShift) continue;
            // move the common zeros: the next shift y -> y + s of both inputs
            bool ok = false;
            while (!ok && sh[i] < kMaxShift) {
                ++sh[i];
                ok = shift_y_i64((const int64_t *)a[i].coef, a[i].deg_x, a[i].deg_y, sh[i], sa[i]) &&
                     shift_y_i64((const int64_t *)b[i].coef, b[i].deg_x, b[i].deg_y, sh[i], sb[i]);
            }
            if (!ok) return c->fail(GBR_EVERIFY, "bivariate gcd: the Kronecker images keep a spurious common factor");
            D[i] = D0[i];
            tries[i] = 0;
        }
        pend.swap(retry);
    }
    return GBR_OK;
}

extern "C" int gbr_gcd2_batch(gbr_ctx *c, int n, const gbr_bipoly *a, const gbr_bipoly *b, gbr_bigbipoly *h,
                              gbr_bigbipoly *a_over_h, gbr_bigbipoly *b_over_h) {
    if (!c || n < 0 || (n && (!a || !b || !h || !a_over_h || !b_over_h))) return GBR_EINVAL;
    if (n == 0) return GBR_OK;
    NvtxScope call("gbr_gcd2_batch");
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

extern "C" int gbr_teissier_res_batch(gbr_ctx *c, int n, const gbr_bipoly *f, gbr_bigpoly *q) {
    if (!c || n < 0 || (n && (!f || !q))) return GBR_EINVAL;
    for (int i = 0; i < n; ++i) q[i] = gbr_bigpoly{-1, 0, nullptr, nullptr};
    if (n == 0) return GBR_OK;
    NvtxScope call("gbr_teissier_res_batch");
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

// ------------------------------------------------------------------ content removal

// content of f with respect to `var` (Section 2, content removal: h = gcd(f_0, f_1,
// ...) of the coefficients of the powers of var, polynomials in the other
// variable): a tree of batched gcds, all inputs of a level in one device batch.
// The gcd of int64 polynomials is read back into int64 for the next level;
// GBR_ELIMIT when a partial gcd does not fit.
static int content_locked(gbr_ctx *c, int n, const gbr_bipoly *f, int var, gbr_bigpoly *out) {
    std::vector<std::vector<std::vector<int64_t>>> level(n);   // per job: its polynomials
    for (int i = 0; i < n; ++i) {
        const gbr_bipoly &p = f[i];
        if (!p.coef || p.deg_x < 0 || p.deg_y < 0 || p.words != 1)
            return c->fail(GBR_EINVAL, "content inputs must be int64 bipolys (words = 1)");
        const int64_t *cf = (const int64_t *)p.coef;
        const int nr = var ? p.deg_y + 1 : p.deg_x + 1, nc = var ? p.deg_x + 1 : p.deg_y + 1;
        for (int r = 0; r < nr; ++r) {
            std::vector<int64_t> row(nc);
            bool any = false;
            for (int k = 0; k < nc; ++k) {
                row[k] = var ? cf[(size_t)r * (p.deg_x + 1) + k] : cf[(size_t)k * (p.deg_x + 1) + r];
                any = any || row[k];
            }
            if (any) level[i].push_back(std::move(row));
        }
        if (level[i].size() == 1) level[i].push_back(level[i][0]);   // gcd(p, p) normalises p
    }
    while (true) {
        std::vector<gbr_upoly> P, Q;
        std::vector<std::pair<int, int>> who;   // (job, slot of the result)
        std::vector<std::vector<std::vector<int64_t>>> next(n);
        for (int i = 0; i < n; ++i) {
            const size_t m = level[i].size();
            if (m < 2) {   // finished (or zero): carried to the next level as it is
                next[i] = level[i];
                continue;
            }
            for (size_t k = 0; k + 1 < m; k += 2) {
                P.push_back(gbr_upoly{(int32_t)level[i][k].size() - 1, 1, level[i][k].data()});
                Q.push_back(gbr_upoly{(int32_t)level[i][k + 1].size() - 1, 1, level[i][k + 1].data()});
                who.push_back({i, (int)next[i].size()});
                next[i].emplace_back();
            }
            if (m % 2) next[i].push_back(level[i][m - 1]);
        }
        if (P.empty()) break;
        std::vector<gbr_bigpoly> g(P.size());
        int st = gbr_gcd_cof_locked(c, (int)P.size(), P.data(), Q.data(), g.data(), nullptr, nullptr);
        if (st) return st;
        int rc = GBR_OK;
        for (size_t t = 0; t < g.size(); ++t) {
            std::vector<int64_t> &dst = next[who[t].first][who[t].second];
            const gbr_bigpoly &b = g[t];
            dst.assign((size_t)std::max(b.deg, 0) + 1, 0);
            for (int k = 0; k <= b.deg && rc == GBR_OK; ++k) {
                uint64_t mag = 0;
                for (int l = 0; l < b.limbs; ++l) {
                    const uint32_t v = b.mag[(size_t)k * b.limbs + l];
                    if (l >= 2 && v) rc = GBR_ELIMIT;
                    if (l < 2) mag |= (uint64_t)v << (32 * l);
                }
                if (mag > (uint64_t)INT64_MAX) rc = GBR_ELIMIT;
                dst[k] = b.sign[k] < 0 ? -(int64_t)mag : (int64_t)mag;
            }
            gbr_free_result(c, &g[t]);
        }
        if (rc) return c->fail(rc, "content: a partial gcd does not fit int64");
        level.swap(next);
    }
    // the remaining polynomial of each job is its content (positive leading coefficient)
    std::vector<gbr_bigpoly> res(n);
    for (int i = 0; i < n; ++i) {
        res[i] = gbr_bigpoly{-1, 2, nullptr, nullptr};
        if (!level[i].empty()) {
            int d = (int)level[i][0].size() - 1;
            while (d >= 0 && !level[i][0][d]) --d;
            res[i].deg = d;
        }
    }
    if (!gbr_alloc_results(res.data(), n)) return c->fail(GBR_ENOMEM, "host result allocation");
    for (int i = 0; i < n; ++i) {
        out[i] = res[i];
        for (int k = 0; k <= res[i].deg; ++k) {
            const int64_t v = level[i][0][k];
            const uint64_t mag = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
            out[i].mag[2 * k] = (uint32_t)mag;
            out[i].mag[2 * k + 1] = (uint32_t)(mag >> 32);
            out[i].sign[k] = (int8_t)((v > 0) - (v < 0));
        }
    }
    return GBR_OK;
}

extern "C" int gbr_content_batch(gbr_ctx *c, int n, const gbr_bipoly *f, int var, gbr_bigpoly *out) {
    if (!c || n < 0 || (n && (!f || !out)) || (var != 0 && var != 1)) return GBR_EINVAL;
    for (int i = 0; i < n; ++i) out[i] = gbr_bigpoly{-1, 0, nullptr, nullptr};
    if (n == 0) return GBR_OK;
    NvtxScope call("gbr_content_batch");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    int st;
    try {
        st = content_locked(c, n, f, var, out);
    } catch (std::bad_alloc &) {
        st = c->fail(GBR_ENOMEM, "host allocation");
    }
    if (st)
        for (int i = 0; i < n; ++i) gbr_free_result(c, &out[i]);
    return st;
}
