// Test harness (CPU): the per-(prime, point) resultant routines of the
// evaluation kernels - the formal-degree recursion res_formal and the register
// form res_chain<N> - run on the host through their host paths.  Reads one case
// per line, "p m n f_0 .. f_m g_0 .. g_n" (residues in [0, p), lowest power
// first, m and n the formal degrees), and prints "formal ok chain": the value of
// res_formal, and for the register shapes (N, N), (N, N-1), (N-1, N) with
// 2 <= N <= 32 whether res_chain accepted the point and its value (else "0 0").
// Built and run by test_host_native.py.
#include <cstdio>
#include <vector>

#include "../../paper_1103_4697_gb300/csrc/gbr_elim.cuh"

using namespace gbr;

// Montgomery constants from their definitions: pinv = -p^-1 mod 2^32 (Newton's
// iteration doubles the correct low bits from p p = 1 mod 8), r1 = 2^32 mod p,
// r2 = 2^64 mod p
static ModP make_modp(uint32_t p) {
    uint32_t inv = p;
    for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
    ModP M;
    M.p = p;
    M.pinv = 0u - inv;
    M.r1 = (uint32_t)((1ull << 32) % p);
    M.r2 = (uint32_t)(((unsigned __int128)1 << 64) % p);
    return M;
}

template <int N>
static uint32_t chain(const std::vector<uint32_t> &f, const std::vector<uint32_t> &g, int m, int n, const ModP &M,
                      bool &ok) {
    uint32_t F[N + 1] = {}, G[N + 1] = {};
    for (int k = 0; k <= m; ++k) F[k] = f[k];
    for (int k = 0; k <= n; ++k) G[k] = g[k];
    return res_chain<N>(F, G, m, n, M, ok);
}

template <int N>
static uint32_t chain_n(int want, const std::vector<uint32_t> &f, const std::vector<uint32_t> &g, int m, int n,
                        const ModP &M, bool &ok) {
    if constexpr (N > 32) {
        ok = false;
        return 0u;
    } else {
        if (want == N) return chain<N>(f, g, m, n, M, ok);
        return chain_n<N + 1>(want, f, g, m, n, M, ok);
    }
}

int main() {
    unsigned p;
    int m, n;
    while (std::scanf("%u %d %d", &p, &m, &n) == 3) {
        const ModP M = make_modp(p);
        std::vector<uint32_t> f(m + 1), g(n + 1);
        for (auto &v : f) {
            unsigned x;
            if (std::scanf("%u", &x) != 1) return 1;
            v = mp_to(x, M);
        }
        for (auto &v : g) {
            unsigned x;
            if (std::scanf("%u", &x) != 1) return 1;
            v = mp_to(x, M);
        }
        // res_formal: columns of stride 1, A[t] = coefficient of y^(m - t); it works in place
        std::vector<uint32_t> A(m + 8, 0u), B(n + 8, 0u);
        for (int t = 0; t <= m; ++t) A[t] = f[m - t];
        for (int t = 0; t <= n; ++t) B[t] = g[n - t];
        const uint32_t formal = mp_from(res_formal(A.data(), m, B.data(), n, 1, M), M);
        const int N = m > n ? m : n;
        const bool reg = N >= 2 && N <= 32 && (m == N || m == N - 1) && (n == N || n == N - 1);
        bool ok = false;
        uint32_t ch = 0u;
        if (reg) ch = mp_from(chain_n<2>(N, f, g, m, n, M, ok), M);
        std::printf("%u %d %u\n", formal, ok ? 1 : 0, ok ? ch : 0u);
    }
    return 0;
}
