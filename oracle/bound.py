"""Coefficient bound of res_y(f, g) by Hadamard's inequality (test infrastructure only).

Section 4 ("Symbolic Speedups") computes resultants by the modular method of
Brown and Collins, which needs primes whose product exceeds twice a bound on
the coefficients of the result; the paper names no bound.  The library plans
its primes with the Hadamard-type bound below, and this module evaluates that
bound from its definition, in exact integer and rational arithmetic, as an
enclosure [lo, hi] of its base-2 logarithm (width 2^-40).  Nothing here uses
floating point.

Definition.  On the unit circle |x| = 1 every coefficient of R(x) = res_y(f, g)
is at most max |R(x)| in absolute value (it is a Fourier coefficient of
R(e^{i theta})).  For a fixed x, R(x) = det S(x) with S the Sylvester matrix
(n rows of f's coefficients, m rows of g's, decreasing powers of y), and
Hadamard's inequality bounds |det S(x)| by the product of the Euclidean norms
of its rows, and by that of its columns.  An entry f_i(x) satisfies
|f_i(x)|^2 <= G(f_i) = A_0 + 2 sum_{k >= 1} |A_k| with A_k = sum_a c_a c_{a+k}
the autocorrelation of f_i's x-coefficients (|f_i(x)|^2 = A_0 + 2 sum_k A_k
cos k theta).  Scaling y -> lambda y multiplies the resultant by lambda^(m n)
and row i of the Sylvester entries by lambda^i, so for every lambda > 0

    |coef R| <= min(rows(lambda), cols(lambda)) / lambda^(m n),

rows(lambda) = prod over the n f-rows of sqrt(sum_i lambda^(2i) G(f_i)) times
prod over the m g-rows of sqrt(sum_j lambda^(2j) G(g_j)), cols(lambda) the
product over the m + n columns of sqrt(sum of lambda^(2 deg) G(entry)).  The
bound is the minimum over the thirteen values log2 lambda in LOG2_LAMBDA; a
column without entries makes the determinant 0 (bound -inf).

Summed forms (small shapes).  For a row or a column with entries h_e scaled by
w_e = lambda^(2 deg e), the squared norm at x = e^{it} is sum_e w_e |h_e(x)|^2 =
C_0 + 2 sum_{k>=1} C_k cos kt with C_k = sum_e w_e A_k(h_e), hence at most
C_0 + 2 sum_k |C_k|: the absolute values taken after the sum over the entries, which
is never more than sum_e w_e G(h_e).  The library evaluates these forms for small
shapes (y-degrees at most SUMMED_MAX_Y, entries of x-degree at most SUMMED_MAX_X,
coefficients below 2^SUMMED_COEF_BITS in magnitude) at lambda = 1 and 2^(1/8), and
the bound is the least of all forms.
"""

from __future__ import annotations

from fractions import Fraction
from math import isqrt

# 4 log2(lambda) for the thirteen scalings: log2 lambda = 0, 1/4, 1/2, 3/4, 1,
# 3/2, 2, 3, 4, 5, 6, -1/2, -1
LOG2_LAMBDA_Q = (0, 1, 2, 3, 4, 6, 8, 12, 16, 20, 24, -2, -4)

_W = 256            # bits kept in the mantissa while squaring
_T = 40             # binary digits of log2 computed
_SQRT2_BITS = 320
_S2_LO = Fraction(isqrt(2 << (2 * _SQRT2_BITS)), 1 << _SQRT2_BITS)   # <= sqrt 2
_S2_HI = _S2_LO + Fraction(1, 1 << _SQRT2_BITS)                       # > sqrt 2


SUMMED_MAX_Y = 24
SUMMED_MAX_X = 24
SUMMED_COEF_BITS = 28
SUMMED_Q8 = (0, 1)       # 8 log2 lambda of the summed forms: lambda = 1 and 2^(1/8)
_Q4 = 320
_R4_LO = Fraction(isqrt(isqrt(2 << (4 * _Q4))), 1 << _Q4)   # <= 2^(1/4)
_R4_HI = _R4_LO + Fraction(1, 1 << _Q4)                       # > 2^(1/4)


def autocorr(row) -> list[int]:
    """A_k = sum_a h_a h_{a+k} for k = 0 .. len(row) - 1."""
    h = [int(c) for c in row]
    L = len(h)
    return [sum(h[a] * h[a + k] for a in range(L - k)) for k in range(L)]


def summed_eligible(F: list, G: list) -> bool:
    """Whether the summed forms apply: y-degrees at most SUMMED_MAX_Y, every entry of
    x-degree at most SUMMED_MAX_X, every coefficient below 2^SUMMED_COEF_BITS."""
    if len(F) - 1 > SUMMED_MAX_Y or len(G) - 1 > SUMMED_MAX_Y:
        return False
    for row in list(F) + list(G):
        nz = [i for i, c in enumerate(row) if c]
        if nz and nz[-1] > SUMMED_MAX_X:
            return False
        if any(abs(int(c)) >= 1 << SUMMED_COEF_BITS for c in row):
            return False
    return True


def _abs_enclosure(I: list) -> tuple[Fraction, Fraction]:
    """[lo, hi] containing |I_0 + I_1 2^(1/4) + I_2 2^(1/2) + I_3 2^(3/4)| for integers I_r."""
    pw = ((Fraction(1), Fraction(1)), (_R4_LO, _R4_HI), (_S2_LO, _S2_HI), (_R4_LO * _S2_LO, _R4_HI * _S2_HI))
    lo = hi = Fraction(0)
    for (a, b), v in zip(pw, I):
        if v >= 0:
            lo, hi = lo + v * a, hi + v * b
        else:
            lo, hi = lo + v * b, hi + v * a
    if lo >= 0:
        return lo, hi
    if hi <= 0:
        return -hi, -lo
    return Fraction(0), max(-lo, hi)


def summed_log2(entries: list, q8: int) -> tuple[Fraction, Fraction]:
    """Enclosure of log2(C_0 + 2 sum_k |C_k|) for entries [(A, deg)] (A the entry's
    autocorrelation) weighted by lambda^(2 deg) = 2^(deg q8 / 4)."""
    K = max(len(A) for A, _ in entries)
    I = [[0, 0, 0, 0] for _ in range(K)]
    for A, d in entries:
        t = d * q8
        for k, a in enumerate(A):
            I[k][t % 4] += a << (t // 4)
    slo, shi = _abs_enclosure(I[0])
    for k in range(1, K):
        lo, hi = _abs_enclosure(I[k])
        slo, shi = slo + 2 * lo, shi + 2 * hi
    return _log2_digits(slo.numerator, slo.denominator, False), _log2_digits(shi.numerator, shi.denominator, True)


def autocorr_g(row) -> int:
    """G(h) = A_0 + 2 sum_{k>=1} |A_k|, A_k = sum_a h_a h_{a+k}: the bound on |h(x)|^2,
    |x| = 1, that the Hadamard product uses for one entry."""
    h = [int(c) for c in row]
    L = len(h)
    g = sum(c * c for c in h)
    for k in range(1, L):
        g += 2 * abs(sum(h[a] * h[a + k] for a in range(L - k)))
    return g


def _log2_digits(num: int, den: int, up: bool) -> Fraction:
    """A lower (up=False) or upper (up=True) bound of log2(num/den), num, den > 0, within
    2^-T: the integer part from the bit lengths, then T binary digits by repeated
    squaring of the mantissa, each square rounded in the bound's direction."""
    e = num.bit_length() - den.bit_length()
    # mantissa y = num / (den 2^e) in [1/2, 2); move it to [1, 2)
    if (num << max(0, -e)) < (den << max(0, e)):
        e -= 1
    # Y ~ y 2^W, rounded in the bound's direction
    sh = _W - e
    if sh >= 0:
        q, r = divmod(num << sh, den)
    else:
        q, r = divmod(num, den << -sh)
    Y = q + (1 if up and r else 0)
    one, two = 1 << _W, 1 << (_W + 1)
    digits = 0
    for _ in range(_T):
        Y = Y * Y
        Y = (Y >> _W) + (1 if up and (Y & (one - 1)) else 0)
        digits <<= 1
        if Y >= two:
            digits |= 1
            Y = (Y >> 1) + (1 if up and (Y & 1) else 0)
    val = Fraction(e) + Fraction(digits, 1 << _T)
    # the squares rounded upward keep the mantissa at most 2 (1 + 2^-200), so the
    # digits still left are at most 2^-T (1 + 2^-199); rounded downward it stays >= 1
    return val + Fraction(2, 1 << _T) if up else val


def log2_interval(a: Fraction, b: Fraction = Fraction(0)) -> tuple[Fraction, Fraction]:
    """[lo, hi] containing log2(a + b sqrt 2) for rationals a, b >= 0, a + b > 0."""
    a, b = Fraction(a), Fraction(b)
    lo = a + b * _S2_LO
    hi = a + b * _S2_HI
    return _log2_digits(lo.numerator, lo.denominator, False), _log2_digits(hi.numerator, hi.denominator, True)


def _scaled(gval: int, deg: int, q: int) -> tuple[Fraction, Fraction]:
    """lambda^(2 deg) G with 4 log2 lambda = q, as a + b sqrt 2: 2^(deg q / 2)."""
    t = deg * q                       # lambda^(2 deg) = 2^(t / 2)
    if t % 2 == 0:
        return Fraction(gval) * Fraction(2) ** (t // 2), Fraction(0)
    return Fraction(0), Fraction(gval) * Fraction(2) ** ((t - 1) // 2)


def hadamard_log2(F: list, G: list, summed: bool = True) -> tuple[Fraction, Fraction] | None:
    """Enclosure [lo, hi] of log2 of the bound for the y-coefficient lists F (f_0..f_m)
    and G (g_0..g_n), each entry a list of x-coefficients, with m, n the y-degrees
    (F[m], G[n] non-zero); None when a Sylvester column is empty (R = 0); (0, 0) when
    m = n = 0 (R = 1).  summed=False leaves out the summed forms (for comparison)."""
    m, n = len(F) - 1, len(G) - 1
    if m <= 0 and n <= 0:
        return Fraction(0), Fraction(0)
    gf = [autocorr_g(r) for r in F]
    gg = [autocorr_g(r) for r in G]
    best_lo = best_hi = None
    for q in LOG2_LAMBDA_Q:
        sf = [_scaled(gf[i], i, q) for i in range(m + 1)]
        sg = [_scaled(gg[j], j, q) for j in range(n + 1)]
        # rows: n copies of f's row norm, m copies of g's
        lo = hi = Fraction(0)
        for s, count in ((sf, n), (sg, m)):
            if count:
                l, h = log2_interval(sum(x[0] for x in s), sum(x[1] for x in s))
                lo += Fraction(count, 2) * l
                hi += Fraction(count, 2) * h
        row = (lo, hi)
        # columns: column c of f-row r holds f_{m - (c - r)} (0 <= c - r <= m), of
        # g-row r holds g_{n - (c - r)}
        clo = chi = Fraction(0)
        empty = False
        for c in range(m + n):
            a = b = Fraction(0)
            for r in range(max(0, c - m), min(n - 1, c) + 1):
                x = sf[m - (c - r)]
                a, b = a + x[0], b + x[1]
            for r in range(max(0, c - n), min(m - 1, c) + 1):
                x = sg[n - (c - r)]
                a, b = a + x[0], b + x[1]
            if a == 0 and b == 0:
                empty = True
                break
            l, h = log2_interval(a, b)
            clo += l / 2
            chi += h / 2
        if empty:
            return None
        lam = Fraction(m * n * q, 4)
        lo_q = min(row[0], clo) - lam
        hi_q = min(row[1], chi) - lam
        best_lo = lo_q if best_lo is None else min(best_lo, lo_q)
        best_hi = hi_q if best_hi is None else min(best_hi, hi_q)
    if summed and summed_eligible(F, G):
        af = [autocorr(r) for r in F]
        ag = [autocorr(r) for r in G]
        for q8 in SUMMED_Q8:
            lo = hi = Fraction(0)
            for A, count in ((af, n), (ag, m)):
                if count:
                    l, h = summed_log2([(A[i], i) for i in range(len(A))], q8)
                    lo += Fraction(count, 2) * l
                    hi += Fraction(count, 2) * h
            clo = chi = Fraction(0)
            for c in range(m + n):
                ents = [(af[m - (c - r)], m - (c - r)) for r in range(max(0, c - m), min(n - 1, c) + 1)]
                ents += [(ag[n - (c - r)], n - (c - r)) for r in range(max(0, c - n), min(m - 1, c) + 1)]
                l, h = summed_log2(ents, q8)
                clo += l / 2
                chi += h / 2
            lam = Fraction(m * n * q8, 8)
            best_lo = min(best_lo, min(lo, clo) - lam)
            best_hi = min(best_hi, min(hi, chi) - lam)
    return best_lo, best_hi


def resultant_bound_log2(f, g) -> tuple[Fraction, Fraction] | None:
    """hadamard_log2 for bivariate rows f[j][i] = coefficient of x^i y^j (zero rows above
    the y-degree ignored); None for a zero input or an empty column."""
    def rows(p):
        r = [[int(c) for c in row] for row in p]
        while r and not any(r[-1]):
            r.pop()
        return r

    F, G = rows(f), rows(g)
    if not F or not G:
        return None
    return hadamard_log2(F, G)


def log2_floor_half_pred(M: int) -> Fraction:
    """A lower bound of log2((M - 1) / 2) for an integer M >= 4: M > 2 B + 1 holds for
    every B with log2 B below it."""
    return _log2_digits(M - 1, 2, False)
