// Test harness (CPU): the planner's routing helpers of gbr_internal.h as the host
// sees them - which shapes take the register form (reg_shape), the evaluation
// point order (point_of), the point sets of the interpolation matrices
// (vinv_point), the padded row count of the residue layout (rows4), the size of a
// root-of-unity point set (root_points), the point-set choice (roots_pay) and the
// shared point counts of a batch (share_point_counts).  Prints
// them for a Python checker.  Built and run by test_host_native.py with the CUDA
// toolkit's include directory (the header declares the launch wrappers).
#include <cstdio>

#include "../../paper_1103_4697_gb300/csrc/gbr_internal.h"

using namespace gbr;

int main() {
    for (int m = 0; m <= 40; ++m)
        for (int n = 0; n <= 40; ++n) std::printf("reg %d %d %d\n", m, n, reg_shape(m, n));
    for (int j = 0; j < 64; ++j)
        std::printf("pt %d %d %d %d %d %d\n", j, point_of(0, j), point_of(1, j), vinv_point(VINV_SYM, j),
                    vinv_point(VINV_EVEN, j), vinv_point(VINV_ODD, j));
    for (int m = 0; m <= 130; ++m) std::printf("rows4 %d %d\n", m, rows4(m));
    for (int P = 1; P <= 16384; P += (P < 1100 ? 1 : 97)) std::printf("rootn %d %d\n", P, root_points(P));
    // the point-set choice for the shapes of the measured crossover: (P, tf, tg, m, n, pairs sharing P)
    const int cases[][6] = {{401, 231, 231, 20, 20, 4096}, {577, 325, 325, 24, 24, 1024}, {257, 153, 153, 16, 16, 1024},
                            {8193, 6147, 6147, 2, 2, 8},   {4097, 2307, 2307, 8, 8, 8},   {1025, 585, 585, 8, 8, 8},
                            {401, 231, 231, 20, 20, 8},    {16001, 12003, 12003, 2, 2, 4000}};
    for (auto &c : cases)
        std::printf("roots %d %d %d %d %d %d %d %d\n", c[0], c[1], c[2], c[3], c[4], c[5],
                    (int)roots_pay(c[0], root_points(c[0]), c[1], c[2], c[3], c[4], c[5], true, true, false),
                    (int)roots_pay(c[0], root_points(c[0]), c[1], c[2], c[3], c[4], c[5], true, false, false));
    // quartic sets: value count, lane pairs and the rows of the quarter parts
    for (int P = 1; P <= 64; ++P)
        std::printf("quad %d %d %d %d %d %d %d %d\n", P, quad_h(P), quad_pe(P), quad_pairs(P), quad_rows(P, 0),
                    quad_rows(P, 1), quad_rows(P, 2), quad_rows(P, 3));
    // shared point counts: a few batches of (point count, pairs)
    const std::vector<std::vector<std::pair<int32_t, int>>> batches = {
        {{61, 6}, {65, 4}, {67, 2}, {71, 4}, {73, 4}},
        {{401, 4096}},
        {{33, 200}, {35, 10}, {37, 10}},
        {{100, 50}, {104, 50}, {106, 50}, {108, 50}},
        {{1000, 3}, {1030, 3}, {1062, 3}, {1070, 3}, {1200, 3}},
        {{5, 1}, {6, 1}, {9, 1}, {10, 1}, {14, 1}},
        {{1020, 8}, {1024, 8}, {1030, 4}, {1050, 4}}};
    for (size_t b = 0; b < batches.size(); ++b) {
        const std::vector<int32_t> to = share_point_counts(batches[b], 128);
        for (size_t i = 0; i < to.size(); ++i)
            std::printf("share %zu %d %d %d\n", b, batches[b][i].first, batches[b][i].second, to[i]);
    }
    return 0;
}
