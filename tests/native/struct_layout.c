/* Test program (CPU): sizeof and the offset of every field of the structures
 * include/gbres.h defines, as seen by a C compiler, one line per structure
 * ("name size field:offset ..."); compared with the Python binding's ctypes
 * layouts by test_host_lib.py. */
#include <stddef.h>
#include <stdio.h>

#include "gbres.h"

#define F(T, f) printf(" " #f ":%zu", offsetof(T, f))

int main(void) {
    printf("BiPoly %zu", sizeof(gbr_bipoly)); F(gbr_bipoly, deg_x); F(gbr_bipoly, deg_y); F(gbr_bipoly, words);
    F(gbr_bipoly, coef); printf("\n");
    printf("UPoly %zu", sizeof(gbr_upoly)); F(gbr_upoly, deg); F(gbr_upoly, words); F(gbr_upoly, coef); printf("\n");
    printf("BigPoly %zu", sizeof(gbr_bigpoly)); F(gbr_bigpoly, deg); F(gbr_bigpoly, limbs); F(gbr_bigpoly, mag);
    F(gbr_bigpoly, sign); printf("\n");
    printf("BigBiPoly %zu", sizeof(gbr_bigbipoly)); F(gbr_bigbipoly, deg_x); F(gbr_bigbipoly, deg_y);
    F(gbr_bigbipoly, c); printf("\n");
    printf("Sqf %zu", sizeof(gbr_sqf)); F(gbr_sqf, unit); F(gbr_sqf, count); F(gbr_sqf, factors); printf("\n");
    printf("Stats %zu", sizeof(gbr_stats)); F(gbr_stats, bounds_ms); F(gbr_stats, reduce_ms); F(gbr_stats, evalres_ms);
    F(gbr_stats, interp_ms); F(gbr_stats, crt_ms); F(gbr_stats, gcd_ms); F(gbr_stats, total_ms); F(gbr_stats, kernels);
    F(gbr_stats, subproblems); F(gbr_stats, modmul); F(gbr_stats, modmul_evalres); F(gbr_stats, h2d_bytes);
    F(gbr_stats, d2h_bytes); F(gbr_stats, dropped_points); F(gbr_stats, dropped_primes); F(gbr_stats, graph_replayed);
    F(gbr_stats, redo_warps); F(gbr_stats, root_pairs); F(gbr_stats, quad_pairs);
    printf("\n");
    printf("Calib %zu", sizeof(gbr_calib)); F(gbr_calib, modmul_per_s); F(gbr_calib, mulsub_per_s);
    F(gbr_calib, sm_clock_mhz); F(gbr_calib, sms); F(gbr_calib, fma3_per_s);
    F(gbr_calib, shoup_per_s); printf("\n");
    printf("ResInfo %zu", sizeof(gbr_res_info)); F(gbr_res_info, m); F(gbr_res_info, n); F(gbr_res_info, deg_bound);
    F(gbr_res_info, primes); F(gbr_res_info, limbs); F(gbr_res_info, log2_bound); printf("\n");
    printf("Job %zu", sizeof(gbr_job)); F(gbr_job, kind); F(gbr_job, var); F(gbr_job, f); F(gbr_job, g); F(gbr_job, p);
    F(gbr_job, q); printf("\n");
    printf("ServeStats %zu", sizeof(gbr_serve_stats)); F(gbr_serve_stats, submitted); F(gbr_serve_stats, completed);
    F(gbr_serve_stats, batches); F(gbr_serve_stats, max_batch); F(gbr_serve_stats, peak_bytes);
    F(gbr_serve_stats, waits_for_memory); printf("\n");
    return 0;
}
