// Test harness (CPU): the choice of the Kronecker candidate in the bivariate gcd
// (kron_shift).  Reads cases from stdin - D, then for G, phi(a)/G and phi(b)/G the
// degree and the sign of every coefficient - and prints the chosen shift per case.
// Built and run by test_host_native.py.
#include <cstdio>
#include <vector>

#include "../../paper_1103_4697_gb300/csrc/gbr_kron.h"

static bool read_poly(std::vector<int8_t> &sg, gbr_bigpoly &p) {
    int deg;
    if (std::scanf("%d", &deg) != 1) return false;
    sg.assign(deg + 1 > 0 ? deg + 1 : 1, 0);
    for (int k = 0; k <= deg; ++k) {
        int v;
        if (std::scanf("%d", &v) != 1) return false;
        sg[k] = (int8_t)v;
    }
    p.deg = deg;
    p.limbs = 1;
    p.mag = nullptr;
    p.sign = sg.data();
    return true;
}

int main() {
    int n;
    if (std::scanf("%d", &n) != 1) return 1;
    for (int i = 0; i < n; ++i) {
        int D;
        if (std::scanf("%d", &D) != 1) return 1;
        std::vector<int8_t> s0, s1, s2;
        gbr_bigpoly g, a, b;
        if (!read_poly(s0, g) || !read_poly(s1, a) || !read_poly(s2, b)) return 1;
        std::printf("%d\n", gbr::kron::kron_shift(g, a, b, D));
    }
    return 0;
}
