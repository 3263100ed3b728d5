/*
 * gbres.h - exact multi-modular resultants and gcds on GB300 (sm_103a).
 *
 * C ABI of libgbres.so.  The library computes, exactly and with integer
 * arithmetic only,
 *
 *   res_y(f, g) in Z[x]   for f, g in Z[x, y]              (gbr_resultant)
 *   res_y(f, df/dy)       the projection resultant R        (gbr_discriminant_res)
 *   gcd(p, q) in Z[x]     for univariate integer polynomials (gbr_gcd)
 *
 * These are the two symbolic operations of Berberich, Emeliyanenko, Kobel and
 * Sagraloff, "Arrangement Computation for Planar Algebraic Curves":
 * Section 2.1 (Projection Phase) computes R = res(f, f_y, y) and its square-free
 * factorisation by gcds; Section 3 (Arrangement Computation) computes
 * R_CD = res(f, g, y); Section 4 (Implementation, "Symbolic Speedups") states
 * that both run on the GPU by the divide-conquer-combine scheme of Brown and
 * Collins: modular and evaluation homomorphisms, independent subproblems over
 * a prime field, then interpolation and Chinese remaindering, and suggests
 * moving the initial modular reduction to the GPU as well.
 *
 * Resultant definition (the value returned): det of the Sylvester matrix of f
 * and g as polynomials in the eliminated variable, with their degrees taken
 * over Z[other variable] (so R vanishes where both leading coefficients
 * vanish, Section 3).  f rows come first, in decreasing powers; hence
 * res(g, f) = (-1)^(mn) res(f, g).  f = 0 or g = 0 gives the zero polynomial;
 * m = n = 0 gives 1.
 *
 * gcd definition: the gcd in Z[x] including the gcd of the integer contents,
 * normalised to a positive leading coefficient; gcd(0, 0) = 0.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Every call returns a status (GBR_OK or an error below) and never aborts.
 * - Inputs are caller-owned and only read during the call.
 * - gbr_bigpoly results are allocated by the library (host memory) and stay
 *   valid until gbr_free_result.
 * - Calls on one context are serialised by the context; use one context per
 *   host thread for concurrency, or the submit/poll serving interface.
 * - On GBR_EDEVICE the CUDA error text is available from gbr_last_error().
 */
#ifndef GBRES_H
#define GBRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define GBR_OK        0
#define GBR_EINVAL    1   /* null pointer, negative extent, words out of range, var not 0/1 */
#define GBR_ENOMEM    2   /* request exceeds the context's device-memory budget, or host malloc failed */
#define GBR_EDEVICE   3   /* a CUDA call failed (text in gbr_last_error) */
#define GBR_ETIMEOUT  4   /* gbr_poll: not finished within timeout_ms */
#define GBR_EAGAIN    5   /* gbr_poll with timeout 0: not finished yet */
#define GBR_EVERIFY   6   /* gcd, square-free: the exact check still failed with every allowed prime */
#define GBR_ELIMIT    7   /* input beyond a documented size limit (see GBR_MAX_*) */
#define GBR_ECANCELED 8   /* serving: the context was shut down before the job ran */
#define GBR_ENOTFOUND 9   /* serving: unknown ticket */

/* ------------------------------------------------------------------ limits */
#define GBR_MAX_WORDS   8     /* 64-bit words per input coefficient (512-bit inputs) */
#define GBR_MAX_YDEG    127   /* degree in the eliminated variable, per polynomial */
#define GBR_MAX_POINTS  16384 /* evaluation points per resultant = x-degree bound + 1 */
#define GBR_MAX_PRIMES  2048  /* primes per result (about 62 000-bit coefficients) */
#define GBR_MAX_UDEG    8191  /* degree of a univariate gcd input */

/* ------------------------------------------------------------------ types */
typedef struct gbr_ctx gbr_ctx;

/* Bivariate integer polynomial, dense.  Coefficient of x^i y^j (0 <= i <= deg_x,
 * 0 <= j <= deg_y) is the two's-complement little-endian integer held in the
 * `words` 64-bit words starting at word (j*(deg_x+1) + i)*words of `coef`.
 * deg_x, deg_y are array extents (>= the actual degrees; zero rows/columns
 * are allowed).  words = 1 is a plain int64 array. */
typedef struct {
    int32_t deg_x, deg_y;
    int32_t words;
    const void *coef;
} gbr_bipoly;

/* Univariate integer polynomial: coefficient of x^i is the two's-complement
 * integer in words [i*words, (i+1)*words) of `coef`. */
typedef struct {
    int32_t deg;
    int32_t words;
    const void *coef;
} gbr_upoly;

/* Exact result in Z[x], sign-magnitude.  deg = -1 for the zero polynomial
 * (mag and sign are then NULL).  Coefficient i has magnitude
 * sum_l mag[i*limbs + l] * 2^(32 l) and sign sign[i] in {-1, 0, +1}.
 * Library-owned: release with gbr_free_result. */
typedef struct {
    int32_t deg;
    int32_t limbs;
    uint32_t *mag;
    int8_t *sign;
} gbr_bigpoly;

/* Counters of the last resultant run (gbr_run_resident or a one-shot/batch
 * resultant call).  Stage times are milliseconds between CUDA events on the
 * context's stream (recorded only with GBR_OPT_STATS = 1; bounds_ms includes
 * the host planning that follows the bounds kernel).  Algorithmic modular
 * multiplications, per (prime, point) subproblem of a pair with y-degrees m, n
 * and T non-zero-capable x-coefficients (sum over rows of row degree + 1):
 * evaluation T, elimination 2 m n; per (pair, prime) with P points:
 * interpolation P (P - 1); per output coefficient with k primes: Garner
 * k (k - 1) / 2.  Bytes are the host<->device copies of the call.  A gcd call
 * (gbr_gcd, gbr_gcd_batch) records gcd_ms (CUDA events around the whole call on
 * the context's stream, including the host work between its stages), total_ms
 * (host wall time), kernels, subproblems ((job, prime) pairs of the modular
 * gcds) and the bytes copied; a square-free call (gbr_squarefree,
 * gbr_squarefree_batch) records the same fields, its subproblems being the
 * (polynomial, prime) pairs of the modular Yun runs and of the exact check. */
typedef struct {
    double bounds_ms, reduce_ms, evalres_ms, interp_ms, crt_ms, gcd_ms, total_ms;
    int64_t kernels;          /* kernels launched */
    int64_t subproblems;      /* (prime, point) subproblems solved */
    int64_t modmul;           /* algorithmic modular multiplications, whole path */
    int64_t modmul_evalres;   /* of the evaluation + elimination stage alone */
    int64_t h2d_bytes, d2h_bytes;
    int64_t dropped_points;   /* GBR_OPT_DROP_UNLUCKY: evaluation points flagged unlucky and replaced */
    int64_t dropped_primes;   /* GBR_OPT_DROP_UNLUCKY: primes skipped because a leading coefficient vanishes */
    int64_t graph_replayed;   /* 1 when the device stages ran as a CUDA graph (GBR_OPT_GRAPH); 2 when
                                 the whole step (bounds, a check of the fresh bounds against those
                                 the plan was made from, stages) ran as one graph with no host
                                 planning in between */
    int64_t redo_warps;       /* GBR_OPT_REGISTER_FORM: warps of 32 subproblems solved again on
                                 shared memory */
    int64_t root_pairs;       /* pairs evaluated at roots of unity and interpolated by an inverse
                                 transform (GBR_OPT_POINTS) */
    int64_t quad_pairs;       /* pairs evaluated on the quartic point set 0, +-a, +-i a and
                                 interpolated by four quarter-size contractions (GBR_OPT_POINTS) */
} gbr_stats;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.
 * mem_budget_bytes: device memory the context may use for scratch and
 *   results; requests that do not fit return GBR_ENOMEM (serving: wait).
 * workspace: NULL, or a caller-owned device allocation of at least
 *   mem_budget_bytes that the context sub-allocates from (the Python binding
 *   passes a torch tensor here); with NULL the library allocates the budget
 *   itself with cudaMalloc at creation.
 * stream: NULL for the legacy default stream, or a cudaStream_t on `device`
 *   on which every kernel and copy of the synchronous calls is issued.
 * Returns GBR_EINVAL (bad arguments), GBR_EDEVICE (CUDA failure, no device). */
int gbr_create(gbr_ctx **ctx, int device, size_t mem_budget_bytes, void *workspace, void *stream);

/* Stop the serving worker (pending jobs finish with GBR_ECANCELED), free all
 * device memory the context allocated, and free the context.  NULL is a no-op. */
void gbr_destroy(gbr_ctx *ctx);

const char *gbr_strerror(int status);
const char *gbr_last_error(gbr_ctx *ctx);

/* Options (gbr_set_option). */
#define GBR_OPT_DROP_UNLUCKY 1   /* 0 (default): evaluation points and primes where a leading
                                    coefficient vanishes are kept and solved with the formal
                                    degrees; 1: they are detected, dropped and replaced by spare
                                    points / the next primes (same result, used to test both) */
#define GBR_OPT_STATS        2   /* 1: record per-stage CUDA-event times (gbr_get_stats) */
#define GBR_OPT_GRAPH        3   /* 1 (default): when a resident batch runs again with an unchanged
                                    plan, its device stages (after the bounds and the plan) are
                                    captured into a CUDA graph once and replayed; from the fourth
                                    run on, the whole step is one graph: the bounds kernel, a
                                    device check that the fresh bounds equal those the plan was
                                    made from, and the stages (which return at once on a mismatch,
                                    after which the call plans again and reruns), with no host
                                    round trip between the bounds and the stages */
#define GBR_OPT_EXTRA_PRIMES 4   /* add this many primes beyond the bound (tests: k+1 == k) */
#define GBR_OPT_INTERP_GEMM  5   /* 1 (default): pairs of a batch that share their number of points
                                    are interpolated by one inverse-Vandermonde contraction per
                                    prime; 0: Newton interpolation for every (pair, prime) */
#define GBR_OPT_INTERP_TC    7   /* 1 (default): the inverse-Vandermonde contractions of up to 256
                                    points run on the tensor cores (bf16 digits, exact fp32 sums);
                                    0: on the integer pipes */
#define GBR_OPT_PIPELINE     8   /* 1 (default): one-shot batches of at least 2048 pairs run in
                                    chunks of 1024 on two internal streams, so that copies and
                                    host work overlap the kernels; 0: one piece */
#define GBR_OPT_REGISTER_FORM 6  /* 1 (default): pairs of shape (N, N), (N, N-1) or (N-1, N) in the
                                    eliminated variable, 2 <= N <= 32, are solved with the
                                    polynomials in registers (warps that meet a vanishing leading
                                    coefficient or a non-normal remainder sequence are solved again
                                    on shared memory); 0: every subproblem on shared memory */
#define GBR_OPT_POINTS       9   /* evaluation points of the resultant (Section 4: the evaluation
                                    and interpolation stages of the modular method; the paper fixes
                                    no point set).  0 (default): chosen per pair: roots of unity
                                    where the estimated cost says so, else the quartic set when its
                                    matrices can be cached, else the symmetric integers;
                                    1: the integers 0, +-1, +-2, ... (interpolation by even and odd
                                    inverse-Vandermonde contractions, or Newton); 2: the N-th roots
                                    of unity modulo each prime, N the power of two
                                    >= max(64, deg_x R + 1) (every table prime is 1 mod 2^14, so
                                    N <= 16384 = GBR_MAX_POINTS), interpolation by an inverse
                                    number-theoretic transform in O(N log N); 3: the quartic set
                                    0, +-a, +-i a (a = 1..ceil(deg_x R / 4), i^2 = -1 mod p): four
                                    quarter-size contractions give R(x) = sum_t x^t R_t(x^4) (half
                                    the multiply-adds of 1), used where its matrices can be
                                    cached (else as 1).  Not used in drop mode
                                    (GBR_OPT_DROP_UNLUCKY).  Results are identical; values outside
                                    0..3: GBR_EINVAL. */
int gbr_set_option(gbr_ctx *ctx, int option, int64_t value);
int gbr_get_stats(gbr_ctx *ctx, gbr_stats *out);

/* ------------------------------------------------------------------ one-shot calls */

/* res_var(f, g): var = 1 eliminates y (res_y, the paper's R_CD), var = 0
 * eliminates x.  Bounds, modular reduction, evaluation, per-(prime, point)
 * resultants, interpolation and Chinese remaindering all run on the device.
 * GBR_EINVAL for more than GBR_MAX_WORDS words per coefficient; GBR_ELIMIT when
 * a degree in var exceeds GBR_MAX_YDEG, the degree bound of the result exceeds
 * GBR_MAX_POINTS - 1, or the coefficient bound needs more than GBR_MAX_PRIMES
 * primes (gbr_resultant_info answers these on the host). */
int gbr_resultant(gbr_ctx *ctx, const gbr_bipoly *f, const gbr_bipoly *g, int var, gbr_bigpoly *out);

/* res_var(f, df/dvar), the projection resultant R of Section 2.1, not divided
 * by the leading coefficient. */
int gbr_discriminant_res(gbr_ctx *ctx, const gbr_bipoly *f, int var, gbr_bigpoly *out);

/* gcd(p, q) in Z[x] (Section 2: content removal; Section 2.1: square-free
 * factorisation).  Modular images over the table primes, Chinese remaindering of
 * the gcd and both cofactors, and an exact norm check that proves the result
 * (on failure more primes are added).  Input coefficients: words must be 1;
 * GBR_ELIMIT for a degree above GBR_MAX_UDEG or a bound that needs more than
 * GBR_MAX_PRIMES primes. */
int gbr_gcd(gbr_ctx *ctx, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *out);

/* ------------------------------------------------------------------ batches */

/* n independent resultants in one pass over the device (pairs of any mixed
 * sizes are bucketed by degree); out[i] receives res_var(f[i], g[i]). */
int gbr_resultant_batch(gbr_ctx *ctx, int n, const gbr_bipoly *f, const gbr_bipoly *g, int var,
                        gbr_bigpoly *out);
int gbr_discriminant_res_batch(gbr_ctx *ctx, int n, const gbr_bipoly *f, int var, gbr_bigpoly *out);
int gbr_gcd_batch(gbr_ctx *ctx, int n, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *out);

/* gcd with cofactors: g[i] = gcd(p[i], q[i]) as gbr_gcd_batch computes it, and
 * p_over_g[i] = p[i] / g[i], q_over_g[i] = q[i] / g[i] exactly (from the same
 * certified lift: the cofactors satisfy p = g * p_over_g and q = g * q_over_g).
 * gcd(0, 0) = 0 has zero cofactors.  All three outputs are library-owned. */
int gbr_gcd_cofactors_batch(gbr_ctx *ctx, int n, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *g,
                            gbr_bigpoly *p_over_g, gbr_bigpoly *q_over_g);

/* Resultants and gcds submitted as one batch (Section 4: the two symbolic
 * operations the algorithm relies on; a workload such as a curve analysis asks
 * for both at once): res_out[i] = res_var(f[i], g[i]) as gbr_resultant_batch
 * computes it and gcd_out[i] = gcd(p[i], q[i]) as gbr_gcd_batch computes it.
 * The gcd batch runs on a private worker stream in a host thread of its own
 * while the resultant batch runs on the context's stream (or its pipeline
 * workers), so their device stages and host planning overlap.  Inputs are
 * caller-owned and read during the call; results are library-owned (free each
 * with gbr_free_result).  On any error both output arrays are left empty
 * (deg = -1) and the first failing half's status is returned; the errors of
 * gbr_resultant_batch and gbr_gcd_batch apply.  nres or ngcd may be 0. */
int gbr_mixed_batch(gbr_ctx *ctx, int nres, const gbr_bipoly *f, const gbr_bipoly *g, int var,
                    gbr_bigpoly *res_out, int ngcd, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *gcd_out);

/* ------------------------------------------------------------------ bivariate gcd, Teissier resultant */

/* An exact polynomial in Z[x, y]: coefficient of x^i y^j at index j (deg_x + 1) + i
 * of c (sign-magnitude limbs as gbr_bigpoly; c.deg + 1 = (deg_x + 1)(deg_y + 1)).
 * deg_y = -1 for the zero polynomial.  Library-owned: gbr_free_bigbipoly. */
typedef struct {
    int32_t deg_x, deg_y;
    gbr_bigpoly c;
} gbr_bigbipoly;
void gbr_free_bigbipoly(gbr_ctx *ctx, gbr_bigbipoly *x);

/* h[i] = gcd(a[i], b[i]) in Z[x, y] (normalised so that the leading coefficient in
 * x of its leading coefficient in y is positive; it includes the gcd of the
 * contents) and the cofactors a[i] / h[i], b[i] / h[i] (Section 2.1 needs
 * h = gcd(f_x, f_y) for the Teissier bound).  Inputs: int64 bipolys (words = 1).
 * Method: Kronecker substitution x^i y^j -> z^(i + j D), D above every x-degree,
 * the certified univariate gcd with cofactors on the device, and the map back;
 * the map-back is exact when deg_x h + deg_x (a / h) < D and likewise for b, which
 * is checked, else D grows by one; after four values of D the inputs are shifted
 * by y -> y + s (s = 1, 2, 3; this moves common zeros such as (1, 1), which every
 * monomial substitution sends to z = 1) and the results shifted back exactly.
 * GBR_EVERIFY when every shift fails (or its int64 inputs would overflow);
 * GBR_ELIMIT when an image would exceed GBR_MAX_UDEG. */
int gbr_gcd2_batch(gbr_ctx *ctx, int n, const gbr_bipoly *a, const gbr_bipoly *b, gbr_bigbipoly *h,
                   gbr_bigbipoly *a_over_h, gbr_bigbipoly *b_over_h);

/* q[i] = Q = res(f_x*, f_y*, y) with h = gcd(f_x, f_y), f_x* = f_x / h, f_y* = f_y / h
 * (Section 2.1, the Teissier bound on the number of distinct roots of f(alpha, y):
 * deg_y f - mult(R, alpha) + mult(Q, alpha)).  Derivatives of the int64 input on the
 * host (GBR_ELIMIT on int64 overflow), h and the cofactors by gbr_gcd2_batch, Q by
 * the resultant path (cofactors of up to GBR_MAX_WORDS words).  Q = 0 when f_x or
 * f_y vanishes. */
int gbr_teissier_res_batch(gbr_ctx *ctx, int n, const gbr_bipoly *f, gbr_bigpoly *q);

/* out[i] = the content of f[i] with respect to var (Section 2, content removal:
 * h = gcd(f_0, f_1, ...) in Z[other variable] of the coefficients f_j of var^j; a
 * non-trivial h marks vertical (var = 1) components), with a positive leading
 * coefficient; zero for f = 0.  Inputs: int64 bipolys (words = 1).  A tree of
 * batched gcds on the device, all curves of a level in one batch; GBR_ELIMIT
 * when a partial gcd does not fit int64. */
int gbr_content_batch(gbr_ctx *ctx, int n, const gbr_bipoly *f, int var, gbr_bigpoly *out);

/* ------------------------------------------------------------------ square-free factorisation */

/* R = unit * prod_{i=1..count} factors[i-1]^i (Section 2.1, Projection Phase:
 * the square-free, pairwise coprime factors r_i of R, from Yun's algorithm).
 * Every factor is primitive with a positive leading coefficient; a multiplicity
 * that does not occur has the factor 1 (degree 0); factors[count-1] has positive
 * degree.  unit is a degree-0 polynomial (the content of R with the sign of its
 * leading coefficient), or deg = -1 when R = 0 (count 0).  A constant R gives
 * unit = R, count 0.  Library-owned: release with gbr_free_sqf. */
typedef struct {
    gbr_bigpoly unit;
    int32_t count;
    gbr_bigpoly *factors;
} gbr_sqf;

/* Square-free factorisation of integer polynomials given in the gbr_bigpoly
 * layout (caller-owned host memory; deg <= GBR_MAX_UDEG; leading zero
 * coefficients are ignored).  Device stages: the coefficients modulo a run of
 * table primes, Yun's algorithm over F_p with one warp per (polynomial, prime),
 * the Garner lift of lc(R) times each monic modular factor over primes that
 * share the degree pattern of largest square-free degree (primes whose product
 * exceeds 2^(deg r_i + 3) ||R||_2), and the exact check R = u prod r_i^i modulo
 * primes whose product exceeds both sides' coefficient bounds.  The host takes
 * the primitive parts (big-integer gcds of the lifted coefficients) and u.  A
 * failed check retries with twice the primes; GBR_EVERIFY once the table is
 * exhausted.  GBR_ELIMIT when a lift needs more primes than the lift kernel
 * holds in shared memory (primes + limbs above 1600: about 810 primes, a
 * factor bound above about 24 000 bits).  On error every out[i] is left empty
 * (count 0, NULL pointers). */
int gbr_squarefree(gbr_ctx *ctx, const gbr_bigpoly *r, gbr_sqf *out);
int gbr_squarefree_batch(gbr_ctx *ctx, int n, const gbr_bigpoly *r, gbr_sqf *out);
void gbr_free_sqf(gbr_ctx *ctx, gbr_sqf *x);

/* Device-resident batches: gbr_upload_pairs copies the inputs into device
 * memory once; gbr_run_resident then runs the whole path (bounds included) on
 * them with results left in device memory; gbr_fetch_resident copies results
 * [first, first+count) back.  disc = 1 computes res(f[i], df[i]/dvar) and
 * ignores g.  The handle owns its device memory until gbr_free_resident. */
typedef struct gbr_resident gbr_resident;
int gbr_upload_pairs(gbr_ctx *ctx, int n, const gbr_bipoly *f, const gbr_bipoly *g, int var, int disc,
                     gbr_resident **out);
int gbr_run_resident(gbr_ctx *ctx, gbr_resident *r);

/* The resultants of an arrangement of n curves (Section 3, curve-pair analysis:
 * every pair of curves C, D needs R_C = res(f_C, d f_C / dy), R_D and R_CD =
 * res(f_C, f_D); an arrangement of n curves needs n(n + 1)/2 of them).  Each
 * curve is uploaded once; the jobs are
 *   q = i                       res_var(f[i], d f[i] / dvar),   0 <= i < n
 *   q = n + pair(i, j)          res_var(f[i], f[j]),            0 <= i < j < n
 * with pair(i, j) = i (2n - i - 1) / 2 + (j - i - 1) (pairs in row-major order).
 * gbr_upload_arrangement makes a resident batch of those n(n + 1)/2 jobs (run
 * and fetch it as above); gbr_arrangement_resultants runs it once and writes
 * out[0 .. n(n + 1)/2).  GBR_ELIMIT when n(n + 1)/2 exceeds 2^29. */
int gbr_upload_arrangement(gbr_ctx *ctx, int n, const gbr_bipoly *f, int var, gbr_resident **out);
int gbr_arrangement_resultants(gbr_ctx *ctx, int n, const gbr_bipoly *f, int var, gbr_bigpoly *out);
int gbr_fetch_resident(gbr_ctx *ctx, gbr_resident *r, int first, int count, gbr_bigpoly *out);
void gbr_free_resident(gbr_ctx *ctx, gbr_resident *r);

void gbr_free_result(gbr_ctx *ctx, gbr_bigpoly *out);

/* ------------------------------------------------------------------ serving */

#define GBR_JOB_RESULTANT 0
#define GBR_JOB_DISC      1
#define GBR_JOB_GCD       2
typedef struct {
    int32_t kind;      /* GBR_JOB_* */
    int32_t var;       /* resultants: eliminated variable */
    gbr_bipoly f, g;   /* resultants (g unused for GBR_JOB_DISC) */
    gbr_upoly p, q;    /* gcd */
} gbr_job;

/* Serving (continuous batching): gbr_submit copies the job and returns at once
 * with a ticket.  A worker thread admits queued jobs while the context's memory
 * budget allows, launches them in device batches on several streams so that
 * batches overlap, and keeps residues on the device until each job's result is
 * copied out.  gbr_poll waits up to timeout_ms (0 = do not wait, <0 = forever)
 * and returns GBR_OK with the result, GBR_EAGAIN/GBR_ETIMEOUT if not finished,
 * or the job's own error.  A ticket is consumed by the first successful poll. */
int gbr_submit(gbr_ctx *ctx, const gbr_job *job, uint64_t *ticket);
int gbr_poll(gbr_ctx *ctx, uint64_t ticket, gbr_bigpoly *out, int timeout_ms);

/* The next finished job in completion order, whichever it is: waits up to
 * timeout_ms (0 = do not wait, <0 = until one finishes) and returns its status
 * (GBR_OK with the result in *out, or the job's own error), its ticket, and in
 * *t_done (may be NULL) the time it finished in seconds on gbr_clock.  The
 * ticket is consumed; tickets already consumed by gbr_poll are skipped.
 * GBR_EAGAIN/GBR_ETIMEOUT when none finished in time, GBR_ENOTFOUND when no job
 * is outstanding. */
int gbr_wait_any(gbr_ctx *ctx, int timeout_ms, uint64_t *ticket, gbr_bigpoly *out, double *t_done);

/* Seconds on the library's monotonic clock (the steady clock of the C++
 * runtime: CLOCK_MONOTONIC on Linux). */
double gbr_clock(void);

/* Serving counters: jobs admitted, batches launched, peak bytes in flight. */
typedef struct {
    int64_t submitted, completed, batches, max_batch, peak_bytes, waits_for_memory;
} gbr_serve_stats;
int gbr_get_serve_stats(gbr_ctx *ctx, gbr_serve_stats *out);

/* ------------------------------------------------------------------ calibration */

/* Measured arithmetic ceilings of this GPU for the library's own Montgomery
 * arithmetic (integer pipes), used as the roofline denominators of the
 * evaluation, elimination and interpolation stages: independent chains (each
 * reads only its own value and fixed multipliers; best of 4, 8 and 16 chains
 * per thread) of one Montgomery multiplication, of the fused two-product
 * multiply-subtract, of the fused three-product reduction and of one Horner
 * step with a fixed multiplier in Shoup's form (the evaluation's step, no
 * reduction), timed with CUDA events on the context's stream.  Results in
 * operations per second (an operation of the fused kinds does two or three
 * modular products); sm_clock_mhz is the clock the driver reports for the
 * device (cudaDevAttrClockRate). */
typedef struct {
    double modmul_per_s;
    double mulsub_per_s;
    double sm_clock_mhz;
    int32_t sms;
    double fma3_per_s;
    double shoup_per_s;
} gbr_calib;
int gbr_calibrate(gbr_ctx *ctx, gbr_calib *out);

/* ------------------------------------------------------------------ allocation-free reconstruction */

/* gbr_crt_noalloc has no counterpart in the paper; it is here for callers that
 * must not allocate device memory when they ask for a result - for example a
 * host that reserves all of its GPU memory up front and forbids allocation
 * afterwards, code running inside another framework's memory pool or
 * allocator callback, or a latency-critical loop that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may cause.  It takes no
 * context, calls no cudaMalloc, cudaFree or other allocating routine, and
 * uses only the buffers the caller passes plus a fixed array that the library
 * declares in device memory (4 MiB, held on every GPU that loads the library
 * until the process exits).
 *
 * What it computes: the signed integers X_c, |X_c| < M/2 with
 * M = p_0 p_1 ... p_{k-1} the first k primes of the table (gbr_prime), whose
 * residues X_c mod p_i are residues[i*stride + c] (normal form, in [0, p_i)),
 * for c = 0..ncoef-1 - the Chinese-remaindering step of the resultant
 * (Garner's mixed-radix digits, symmetric lift).  Output: magnitudes in
 * mag[c*limbs + l] (32-bit limbs, least significant first) and signs in
 * sign[c] in {-1, 0, +1}, the layout of gbr_bigpoly.  All four pointers are
 * device memory owned by the caller.
 *
 * Limits: 1 <= k <= GBR_NOALLOC_MAX_PRIMES, ncoef * k <= 1048576 (the fixed
 * array holds one digit per coefficient and prime); beyond them the call
 * returns GBR_ELIMIT without launching anything.  limbs must be at least
 * ceil(31 k / 32) (GBR_EINVAL otherwise); stride >= ncoef.
 *
 * Behaviour: asynchronous on `stream` (NULL: the legacy default stream);
 * results are ready when the stream reaches that point.  The first call on a
 * device, with that device current, looks up the device address of the fixed
 * array (cudaGetSymbolAddress).  CUDA loads a library's device code lazily by
 * default, so that first call is also when the 4 MiB array is mapped on the
 * device: make it before the caller reserves the rest of its device memory
 * (a device with no room left then gets GBR_EDEVICE) and before any stream
 * capture begins.  Every call uses the same fixed array and leaves its last
 * contents there; calls whose kernels overlap on the GPU (other streams, other
 * host threads) overwrite each other's digits and give wrong results, so
 * serialise them.  Returns GBR_EDEVICE if the lookup or the launch fails. */
#define GBR_NOALLOC_MAX_PRIMES 64
int gbr_crt_noalloc(const uint32_t *residues, int k, int ncoef, int64_t stride, uint32_t *mag, int limbs,
                    int8_t *sign, void *stream);

/* ------------------------------------------------------------------ host-side information */

/* The fixed table of primes used by every context: p_0 > p_1 > ... are the
 * largest primes below 2^32 / 3 that are 1 mod 2^14 (30.0 to 30.4 bits each:
 * three products of residues fit one Montgomery reduction, and each prime has
 * roots of unity of order up to 2^14 for GBR_OPT_POINTS).  Host only. */
int gbr_num_primes(void);
int gbr_prime(int index, uint32_t *p);

/* Number of primes from the table whose product exceeds 2^bits (the count a
 * resultant whose coefficients satisfy |c| < 2^(bits-1) needs); -1 when the
 * product of all GBR_MAX_PRIMES primes does not. */
int gbr_primes_for_bits(double bits);

/* Resultant planning for a pair given on the host: actual degrees m, n, the
 * x-degree bound D (min of n deg_x f + m deg_x g and the total-degree Bezout
 * bound), log2 of the Hadamard bound B on |coefficients| and the number of
 * primes k with prod p > 2B + 1 (-1 when more than GBR_MAX_PRIMES would be
 * needed: a resultant call then returns GBR_ELIMIT).  Host only.  disc = 1 uses
 * g = df/dvar.  GBR_ELIMIT when m or n exceeds GBR_MAX_YDEG, GBR_EINVAL for an
 * input of more than GBR_MAX_WORDS words per coefficient.
 * B is the smallest scaled bound over all lambda values; the device evaluates
 * the same bounds in single precision rounded upward, so its B can be slightly
 * larger (at most a few thousandths of a bit) and, in a near tie, take one
 * prime more. */
typedef struct {
    int32_t m, n, deg_bound, primes, limbs;
    double log2_bound;
} gbr_res_info;
int gbr_resultant_info(const gbr_bipoly *f, const gbr_bipoly *g, int var, int disc, gbr_res_info *out);

/* The plan the device made for jobs [first, first + count) of a resident batch
 * in its last gbr_run_resident: actual degrees, x-degree bound of the result
 * (deg_bound; the run may interpolate at more points than deg_bound + 1 when jobs of
 * the batch with close degree bounds share one point count, the coefficients above
 * deg_bound then being 0), primes used (including GBR_OPT_EXTRA_PRIMES), output limbs, and
 * the log2 of the coefficient bound computed on the device (an upper bound of
 * the same scaled Hadamard bound gbr_resultant_info evaluates, in single
 * precision with directed rounding).  A zero result has deg_bound = -1 and
 * primes = 0.  GBR_EINVAL before the first run. */
int gbr_resident_plan(gbr_ctx *ctx, gbr_resident *r, int first, int count, gbr_res_info *out);

#ifdef __cplusplus
}
#endif
#endif /* GBRES_H */
