/* Test program (CPU): include/gbres.h compiled as plain C99 and libgbres.so
 * linked from C, calling the host-only entry points (prime table, prime counts,
 * the resultant plan, status strings).  Prints one line per check; built and
 * run by test_host_lib.py. */
#include <stdint.h>
#include <stdio.h>

#include "gbres.h"

int main(void) {
    uint32_t p0 = 0, p1 = 0;
    int64_t f[] = {-25, 0, 1, 0, 0, 0, 1, 0, 0};   /* x^2 + y^2 - 25: deg_x 2, deg_y 2 */
    int64_t g[] = {-1, 1, 1, 0};                   /* y + x - 1: deg_x 1, deg_y 1 */
    gbr_bipoly F, G;
    gbr_res_info info;
    int st;

    F.deg_x = 2;
    F.deg_y = 2;
    F.words = 1;
    F.coef = f;
    G.deg_x = 1;
    G.deg_y = 1;
    G.words = 1;
    G.coef = g;
    printf("num_primes %d\n", gbr_num_primes());
    st = gbr_prime(0, &p0);
    st |= gbr_prime(1, &p1);
    printf("primes %d %u %u\n", st, (unsigned)p0, (unsigned)p1);
    printf("primes_for_bits %d %d\n", gbr_primes_for_bits(100.0), gbr_primes_for_bits(1.0e9));
    st = gbr_resultant_info(&F, &G, 1, 0, &info);
    printf("info %d %d %d %d %d\n", st, info.m, info.n, info.deg_bound, info.primes);
    st = gbr_resultant_info(&F, NULL, 1, 1, &info);
    printf("disc %d %d %d %d\n", st, info.m, info.n, info.deg_bound);
    printf("bad_var %d\n", gbr_resultant_info(&F, &G, 2, 0, &info));
    printf("strerror %s\n", gbr_strerror(GBR_ELIMIT));
    return 0;
}
