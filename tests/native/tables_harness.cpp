// Test harness (CPU): the host-built constant tables of libgbres - the first K
// table primes with their Montgomery constants, the Garner prefix table, the
// inverse table and the warp Chinese remaindering table - printed for a Python checker (linked against libgbres.so).
// Built and run by test_host_native.py.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1103_4697_gb300/csrc/gbr_internal.h"

int main(int argc, char **argv) {
    const int K = argc > 1 ? std::atoi(argv[1]) : 40, T = argc > 2 ? std::atoi(argv[2]) : 300;
    const ModP *M = gbr::host_mods();
    std::printf("%d\n", gbr::num_primes());
    for (int i = 0; i < K; ++i) std::printf("%u %u %u %u\n", M[i].p, M[i].pinv, M[i].r1, M[i].r2);
    std::vector<uint32_t> g((size_t)K + (size_t)K * (K - 1) / 2), inv((size_t)K * T);
    gbr::garner_prefix_table(K, g.data());
    gbr::inverse_table(K, T, inv.data());
    for (uint32_t v : g) std::printf("%u ", v);
    std::printf("\n");
    for (uint32_t v : inv) std::printf("%u ", v);
    std::printf("\n");
    std::vector<uint32_t> w(gbr::crt_warp_words(K));
    gbr::crt_warp_table(K, w.data());
    std::printf("%d\n", gbr::crt_warp_limbs(K));
    for (uint32_t v : w) std::printf("%u ", v);
    std::printf("\n");
    return 0;
}
