// Test harness (CPU): the planner's routing helpers of gbr_internal.h as the host
// sees them - which shapes take the register form (reg_shape), the evaluation
// point order (point_of), the point sets of the interpolation matrices
// (vinv_point) and the padded row count of the residue layout (rows4).  Prints
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
    return 0;
}
