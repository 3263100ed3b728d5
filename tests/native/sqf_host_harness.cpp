// Test harness (CPU): the square-free path's host helpers - primitive parts of
// lifted factors (with and without a large planted content) and the coefficient
// norms rounded up - on seeded random polynomials; prints inputs and results for
// a Python checker.  Built and run by test_host_native.py.
#include <cstdio>
#include <random>

#include "../../paper_1103_4697_gb300/csrc/gbr_sqf_host.h"

using namespace gbr;
using namespace gbr::sqfh;

int main(int argc, char **argv) {
    const int N = argc > 1 ? std::atoi(argv[1]) : 1000;
    std::mt19937_64 rng(7);
    bn::Scratch S;
    std::printf("%d\n", N);
    for (int it = 0; it < N; ++it) {
        const int d = (int)(rng() % 9);
        int LL = 1 + (int)(rng() % 5);
        std::vector<uint32_t> x((size_t)(d + 1) * LL, 0u);
        std::vector<int8_t> sg(d + 1, 0);
        for (int t = 0; t <= d; ++t) {
            if (t < d && rng() % 4 == 0) continue;   // zero coefficients
            const int nl = 1 + (int)(rng() % LL);
            for (int l = 0; l < nl; ++l) x[(size_t)t * LL + l] = (uint32_t)rng();
            sg[t] = (rng() & 1) ? 1 : -1;
            if (bn::top(&x[(size_t)t * LL], LL) == 0) sg[t] = 0;
        }
        if (sg[d] == 0) {
            x[(size_t)d * LL] = 1u;
            sg[d] = 1;
        }
        if (it % 2 == 0) {   // a planted content of 1 to 3 limbs
            bn::Limbs k(1 + rng() % 3);
            for (auto &v : k) v = (uint32_t)rng();
            if (k.back() == 0) k.back() = 1u;
            const int L2 = LL + (int)k.size();
            std::vector<uint32_t> y((size_t)(d + 1) * L2, 0u);
            for (int t = 0; t <= d; ++t) {
                bn::Limbs c(x.begin() + (size_t)t * LL, x.begin() + (size_t)(t + 1) * LL);
                c.resize(bn::top(c.data(), c.size()));
                const bn::Limbs p = bn::mul_mag(c, k);
                std::copy(p.begin(), p.end(), y.begin() + (size_t)t * L2);
            }
            x.swap(y);
            LL = L2;
        }
        std::printf("%d %d\n", d, LL);
        for (int t = 0; t <= d; ++t) {
            std::printf("%d", sg[t]);
            for (int l = 0; l < LL; ++l) std::printf(" %u", x[(size_t)t * LL + l]);
            std::printf("\n");
        }
        FlatPoly f;
        const bool ok = primitive_part(x.data(), sg.data(), d, LL, f, S);
        std::printf("%d %d\n", (int)ok, f.L);
        if (ok)
            for (int t = 0; t <= d; ++t) {
                std::printf("%d", f.sign[t]);
                for (int l = 0; l < f.L; ++l) std::printf(" %u", f.mag[(size_t)t * f.L + l]);
                std::printf("\n");
            }
        const Norms nr = log2_norms(d + 1, [&](int t, const uint32_t *&p, size_t &n) {
            p = &x[(size_t)t * LL];
            n = sg[t] ? bn::top(p, LL) : 0;
        });
        std::printf("%.17g %.17g %.17g\n", nr.l1, nr.l2, nr.linf);
    }
    return 0;
}
