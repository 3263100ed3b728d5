// Test harness (CPU): the Montgomery arithmetic of the kernels (gbr_modarith.cuh)
// through its host paths, on residues at the ends of their documented ranges.
// Reads "op p args..." lines and prints one result per line, for a Python
// checker with plain modular integer arithmetic.  Built and run by
// test_host_native.py.
//   mul p a b            mp_mul(a, b)               = a b R^-1 mod p  (R = 2^32)
//   mulsub p a x b y     mp_mulsub(a, x, b, y)      = (a x - b y) R^-1 mod p
//   fma2 p a x b y       mp_fma2(a, x, b, y)        = (a x + b y) R^-1 mod p
//   fma3 p a x b y c z   mp_fma3(...)               = (a x + b y + c z) R^-1 mod p
//   to p v / from p x    Montgomery form of any 32-bit v / normal form of x
//   pow p x e / inv p x  in Montgomery form, printed in normal form
//   words p W w_0..w_W-1 mp_from_words: the two's-complement integer mod p (normal form)
#include <cstdio>
#include <cstring>

#include "../../paper_1103_4697_gb300/csrc/gbr_modarith.cuh"

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

int main() {
    char op[16];
    unsigned p;
    while (std::scanf("%15s %u", op, &p) == 2) {
        const ModP M = make_modp(p);
        unsigned a, x, b, y, c, z;
        if (!std::strcmp(op, "mul") && std::scanf("%u %u", &a, &b) == 2) {
            std::printf("%u\n", mp_mul(a, b, M));
        } else if (!std::strcmp(op, "mulsub") && std::scanf("%u %u %u %u", &a, &x, &b, &y) == 4) {
            std::printf("%u\n", mp_mulsub(a, x, b, y, M));
        } else if (!std::strcmp(op, "fma2") && std::scanf("%u %u %u %u", &a, &x, &b, &y) == 4) {
            std::printf("%u\n", mp_fma2(a, x, b, y, M));
        } else if (!std::strcmp(op, "fma3") && std::scanf("%u %u %u %u %u %u", &a, &x, &b, &y, &c, &z) == 6) {
            std::printf("%u\n", mp_fma3(a, x, b, y, c, z, M));
        } else if (!std::strcmp(op, "to") && std::scanf("%u", &a) == 1) {
            std::printf("%u\n", mp_to(a, M));
        } else if (!std::strcmp(op, "from") && std::scanf("%u", &a) == 1) {
            std::printf("%u\n", mp_from(a, M));
        } else if (!std::strcmp(op, "pow") && std::scanf("%u %u", &a, &b) == 2) {
            std::printf("%u\n", mp_from(mp_pow(mp_to(a, M), b, M), M));
        } else if (!std::strcmp(op, "inv") && std::scanf("%u", &a) == 1) {
            std::printf("%u\n", mp_from(mp_inv(mp_to(a, M), M), M));
        } else if (!std::strcmp(op, "words")) {
            int W;
            unsigned long long w[8];
            if (std::scanf("%d", &W) != 1 || W < 1 || W > 8) return 1;
            for (int i = 0; i < W; ++i)
                if (std::scanf("%llu", &w[i]) != 1) return 1;
            std::printf("%u\n", mp_from(mp_from_words((const uint64_t *)w, W, M), M));
        } else {
            return 1;
        }
    }
    return 0;
}
