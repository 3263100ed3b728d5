// Test harness (CPU): the host helpers of the bivariate gcd and the Teissier
// resultant - the int64 shift y -> y + s, the big-integer shift back, the partial
// derivatives and the conversion of sign-magnitude coefficients to
// two's-complement words.  Reads one command per line from stdin and prints one
// result line per command.  Built and run by test_host_native.py.
//
//   S dx dy s c...                      -> "OK c..." | "OVF"
//   U dx dy s (sign nlimbs limb...)...  -> "sign nlimbs limb..." per coefficient
//   D wx dx dy c...                     -> "OK ox oy c..." | "OVF"
//   W dx dy L (sign limb x L)...        -> "OK words w..." | "LIMIT"   (dy = -1: zero)
#include <cstdio>
#include <vector>

#include "../../paper_1103_4697_gb300/csrc/gbr_kron.h"

using namespace gbr;

int main() {
    char op[4];
    while (std::scanf("%3s", op) == 1) {
        if (op[0] == 'S') {
            int dx, dy, s;
            if (std::scanf("%d %d %d", &dx, &dy, &s) != 3) return 1;
            std::vector<int64_t> in((size_t)(dx + 1) * (dy + 1)), out;
            for (auto &v : in)
                if (std::scanf("%lld", (long long *)&v) != 1) return 1;
            if (!kron::shift_y_i64(in.data(), dx, dy, s, out)) {
                std::printf("OVF\n");
                continue;
            }
            std::printf("OK");
            for (int64_t v : out) std::printf(" %lld", (long long)v);
            std::printf("\n");
        } else if (op[0] == 'U') {
            int dx, dy, s;
            if (std::scanf("%d %d %d", &dx, &dy, &s) != 3) return 1;
            std::vector<bn::Big> g((size_t)(dx + 1) * (dy + 1));
            for (auto &b : g) {
                int sg, nl;
                if (std::scanf("%d %d", &sg, &nl) != 2) return 1;
                std::vector<uint32_t> l(nl > 0 ? nl : 1, 0u);
                for (int k = 0; k < nl; ++k)
                    if (std::scanf("%u", &l[k]) != 1) return 1;
                if (sg) b = bn::from_limbs(l.data(), nl, sg);
            }
            kron::unshift_y_big(g, dx, dy, s);
            for (size_t t = 0; t < g.size(); ++t) {
                std::printf("%d %zu", g[t].s, g[t].m.size());
                for (uint32_t v : g[t].m) std::printf(" %u", v);
                std::printf(t + 1 < g.size() ? " " : "\n");
            }
        } else if (op[0] == 'D') {
            int wx, dx, dy;
            if (std::scanf("%d %d %d", &wx, &dx, &dy) != 3) return 1;
            std::vector<int64_t> in((size_t)(dx + 1) * (dy + 1)), buf;
            for (auto &v : in)
                if (std::scanf("%lld", (long long *)&v) != 1) return 1;
            gbr_bipoly f{dx, dy, 1, in.data()}, out{};
            if (!kron::derive(f, wx != 0, buf, out)) {
                std::printf("OVF\n");
                continue;
            }
            std::printf("OK %d %d", out.deg_x, out.deg_y);
            for (size_t t = 0; t < (size_t)(out.deg_x + 1) * (out.deg_y + 1); ++t)
                std::printf(" %lld", (long long)((const int64_t *)out.coef)[t]);
            std::printf("\n");
        } else if (op[0] == 'W') {
            int dx, dy, L;
            if (std::scanf("%d %d %d", &dx, &dy, &L) != 3) return 1;
            const int nco = dy < 0 ? 0 : (dx + 1) * (dy + 1);
            std::vector<uint32_t> mag((size_t)(nco > 0 ? nco : 1) * L, 0u);
            std::vector<int8_t> sign(nco > 0 ? nco : 1, 0);
            for (int t = 0; t < nco; ++t) {
                int sg;
                if (std::scanf("%d", &sg) != 1) return 1;
                sign[t] = (int8_t)sg;
                for (int l = 0; l < L; ++l)
                    if (std::scanf("%u", &mag[(size_t)t * L + l]) != 1) return 1;
            }
            gbr_bigbipoly x;
            x.deg_x = dy < 0 ? -1 : dx;
            x.deg_y = dy;
            x.c = gbr_bigpoly{nco - 1, L, mag.data(), sign.data()};
            std::vector<uint64_t> buf;
            gbr_bipoly out{};
            if (!kron::to_words(x, buf, out)) {
                std::printf("LIMIT\n");
                continue;
            }
            std::printf("OK %d %d %d", out.deg_x, out.deg_y, out.words);
            for (size_t t = 0; t < (size_t)(out.deg_x + 1) * (out.deg_y + 1) * out.words; ++t)
                std::printf(" %llu", (unsigned long long)((const uint64_t *)out.coef)[t]);
            std::printf("\n");
        } else {
            return 1;
        }
    }
    return 0;
}
