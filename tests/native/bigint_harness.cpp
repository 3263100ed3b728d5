// Test harness (CPU): exercises the host big-integer routines of the square-free
// path (long division, Lehmer's gcd, gcd_into) on seeded random operands and prints
// operands and results for a Python checker.  Built and run by test_host_native.py.
#include <cstdio>
#include <random>

#include "../../paper_1103_4697_gb300/csrc/gbr_bigint.h"

using namespace gbr::bn;

static void put(const Limbs &a) {
    std::printf("%zu", a.size());
    for (uint32_t x : a) std::printf(" %u", x);
    std::printf("\n");
}

static Limbs rnd(std::mt19937_64 &r, int n) {
    Limbs a(n);
    for (auto &x : a) x = (uint32_t)r();
    if (r() % 5 == 0)
        for (int i = 0; i < n / 2; ++i) a[i] = 0;   // runs of zero limbs
    if (r() % 7 == 0 && n) a.back() = 0xFFFFFFFFu;  // top limb all ones
    a.resize(top(a.data(), a.size()));
    return a;
}

// operands of 1 to 5 limbs from boundary words (0, 1, 2^31 - 1, 2^31, all ones,
// random): the double-word division path and both sides of its 4-limb limit
static Limbs small(std::mt19937_64 &r) {
    static const uint32_t words[] = {0u, 1u, 0x7FFFFFFFu, 0x80000000u, 0xFFFFFFFFu};
    Limbs a(1 + r() % 5);
    for (auto &x : a) x = r() % 3 ? words[r() % 5] : (uint32_t)r();
    a.resize(top(a.data(), a.size()));
    return a;
}

int main(int argc, char **argv) {
    const int N = argc > 1 ? std::atoi(argv[1]) : 1500;
    const int M = argc > 2 ? std::atoi(argv[2]) : 0;   // small-operand cases after the N others
    std::mt19937_64 rng(20261203);
    Scratch S;
    std::printf("%d\n", N + M);
    for (int it = 0; it < N + M; ++it) {
        Limbs a = rnd(rng, 1 + (int)(rng() % 40)), b = rnd(rng, 1 + (int)(rng() % 40));
        if (it >= N) {
            a = small(rng);
            b = it % 7 == 0 ? a : small(rng);
        }
        switch (it < N ? it % 5 : -1) {
            case 1: {   // a large common factor
                Limbs g = rnd(rng, 1 + (int)(rng() % 20));
                if (!g.empty()) {
                    a = mul_mag(a, g);
                    b = mul_mag(b, g);
                }
                break;
            }
            case 2: b = a; break;                                    // equal operands
            case 3: b = mul_mag(a, rnd(rng, 1 + (int)(rng() % 3))); break;   // a multiple
            case 4: a = rnd(rng, 30); b = rnd(rng, 2); break;       // a huge quotient
            default: break;
        }
        if (a.empty()) a = {7};
        if (b.empty()) b = {5};
        put(a);
        put(b);
        Limbs q, r;
        divmod_mag(a, b, q, r, S);
        put(q);
        put(r);
        Limbs x = a, y = b;
        gcd_lehmer(x, y, S);
        put(x);
        Limbs g = a;
        gcd_into(g, b.data(), b.size(), S);
        put(g);
    }
    return 0;
}
