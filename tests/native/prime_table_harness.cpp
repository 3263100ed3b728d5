// Test harness (CPU): the bytes of the device prime table as the host builds them
// (build_prime_table, linked from libgbres.so) - the (R^3, R^4) pairs of the first
// primes and the Chinese-remaindering tables of the first kCrtFastK primes (Garner
// rows, prefix-product limbs, first non-zero columns) and the root-of-unity
// power tables - printed for a Python checker.  Built and run by test_host_native.py.
#include <cstdio>
#include <vector>

#include "../../paper_1103_4697_gb300/csrc/gbr_internal.h"

using namespace gbr;

int main() {
    std::vector<char> buf;
    build_prime_table(buf);
    const int NP = num_primes();
    const ModP *m = (const ModP *)buf.data();
    const uint2 *r34 = (const uint2 *)(m + NP);
    const uint32_t *tab = (const uint32_t *)(r34 + NP);
    std::printf("%d %zu\n", NP, buf.size());
    for (int i = 0; i < kCrtFastK; ++i) std::printf("%u %u %u\n", m[i].p, r34[i].x, r34[i].y);
    for (int i = 0; i < kCrtGdWords; ++i) std::printf("%u ", tab[i]);
    std::printf("\n");
    for (int l = 0; l < kCrtFastL; ++l) {
        for (int i = 0; i <= kCrtFastK; ++i) std::printf("%u ", tab[kCrtGdWords + l * kCrtFastRow + i]);
        std::printf("\n");
    }
    for (int l = 0; l < kCrtFastL; ++l) std::printf("%u ", tab[kCrtGdWords + kCrtFastL * kCrtFastRow + l]);
    std::printf("\n");
    // root-of-unity tables of the first kCrtFastK primes, then of the last two (with their prime)
    const uint32_t *rt = tab + kCrtTabWords;
    for (int i = 0; i < kCrtFastK + 2; ++i) {
        const int q = i < kCrtFastK ? i : NP - 2 + (i - kCrtFastK);
        if (i >= kCrtFastK) std::printf("%u ", m[q].p);
        for (int j = 0; j < kRootTabWords; ++j) std::printf("%u ", rt[(size_t)q * kRootTabWords + j]);
        std::printf("\n");
    }
    return 0;
}
