"""Pins for the CPU oracle (no GPU).

The oracle is checked against facts that do not come from itself: hand-derived
values, closed forms for planted roots, the symmetry and multiplicativity of the
resultant, a planted common factor, brute-force permutation expansion on tiny
inputs, and sympy where it is installed.  Each check is chosen so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails one of
them.
"""

import json
import math
import os
import random

import pytest

import oracle as O
from oracle.resultant import as_zxy
from paper_1103_4697_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "hand_examples.json")))

RES_METHODS = {
    "bareiss": O.res_bareiss,
    "subres": O.res_subres,
    "evalz": O.res_evalz,
}


def _prod_zx(polys):
    out = (1,)
    for p in polys:
        out = O.zx_mul(out, p)
    return out


def _rand_bipoly(rng, m, dx, lo=-3, hi=3):
    return [[rng.randint(lo, hi) for _ in range(dx + 1)] for _ in range(m + 1)]


def _zx_pow(p, e):
    out = (1,)
    for _ in range(e):
        out = O.zx_mul(out, p)
    return out


# --------------------------------------------------------------------------- hand-derived values


@pytest.mark.parametrize("method", sorted(RES_METHODS))
@pytest.mark.parametrize("k", range(len(GOLD["resultants"])))
def test_hand_resultants(method, k):
    e = GOLD["resultants"][k]
    assert RES_METHODS[method](e["f"], e["g"]) == tuple(e["res"])


@pytest.mark.parametrize("k", range(len(GOLD["res_at_formal"])))
def test_hand_res_at_formal_degree(k):
    e = GOLD["res_at_formal"][k]
    assert O.res_at(e["f"], e["g"], e["a"]) == e["value"]


@pytest.mark.parametrize("k", range(len(GOLD["gcds"])))
def test_hand_gcds(k):
    e = GOLD["gcds"][k]
    assert O.gcd_z(e["p"], e["q"]) == tuple(e["gcd"])


@pytest.mark.parametrize("k", range(len(GOLD["teissier"])))
def test_hand_teissier(k):
    """Hand-derived h, f_x/h, f_y/h and Q (Section 2.1); the first two have
    deg_y(f_x/h) = deg_y(f_y/h) = 1, so swapped operands would flip the sign of Q."""
    from oracle.bigcd import teissier_parts, teissier_q

    e = GOLD["teissier"][k]
    h, fxs, fys = teissier_parts(e["f"])
    assert h == [tuple(r) for r in e["h"]]
    assert fxs == [tuple(r) for r in e["fx_star"]] and fys == [tuple(r) for r in e["fy_star"]]
    assert teissier_q(e["f"]) == tuple(e["q"])


# --------------------------------------------------------------------------- closed forms


@pytest.mark.parametrize("seed,m,n", [(1, 1, 1), (2, 2, 3), (3, 3, 2), (4, 4, 4), (5, 1, 5), (6, 5, 3)])
def test_planted_roots_closed_form(seed, m, n):
    f, g, al, be, a, b = W.planted_roots_pair(seed, m, n)
    diffs = [(ai[0] - bj[0], ai[1] - bj[1]) for ai in al for bj in be]
    want = O.zx_mul((a ** n * b ** m,), _prod_zx([O.zx_trim(d) for d in diffs]))
    for name, fn in RES_METHODS.items():
        assert fn(f, g) == want, name
    if m + n <= 7:
        assert O.res_leibniz(f, g) == want


@pytest.mark.parametrize("seed,m", [(11, 2), (12, 3), (13, 4), (14, 5)])
def test_disc_closed_form(seed, m):
    """f = a prod (y - alpha_i): res(f, f_y) = a^(2m-1) prod_{i != j} (alpha_i - alpha_j)."""
    f, _, al, _, a, _ = W.planted_roots_pair(seed, m, 1)
    diffs = [O.zx_trim((ai[0] - aj[0], ai[1] - aj[1])) for i, ai in enumerate(al)
             for j, aj in enumerate(al) if i != j]
    want = O.zx_mul((a ** (2 * m - 1),), _prod_zx(diffs))
    for method in ("subres", "bareiss", "evalz"):
        assert O.disc_res(f, method) == want


# --------------------------------------------------------------------------- invariants


@pytest.mark.parametrize("seed", range(8))
def test_symmetry(seed):
    rng = random.Random(seed)
    m, n = rng.randint(1, 4), rng.randint(1, 4)
    f = _rand_bipoly(rng, m, rng.randint(0, 3))
    g = _rand_bipoly(rng, n, rng.randint(0, 3))
    f[-1][0] = f[-1][0] or 1
    g[-1][0] = g[-1][0] or 1
    mm, nn = O.ydeg(f), O.ydeg(g)
    for fn in RES_METHODS.values():
        r1, r2 = fn(f, g), fn(g, f)
        assert r2 == (r1 if (mm * nn) % 2 == 0 else O.zx_neg(r1))


@pytest.mark.parametrize("seed", range(6))
def test_multiplicativity(seed):
    rng = random.Random(100 + seed)
    f1 = _rand_bipoly(rng, rng.randint(1, 3), 2)
    f2 = _rand_bipoly(rng, rng.randint(1, 2), 2)
    g = _rand_bipoly(rng, rng.randint(1, 3), 2)
    for p in (f1, f2, g):
        p[-1][0] = p[-1][0] or 2
    f12 = W._mul2(f1, f2)
    for fn in (O.res_subres, O.res_bareiss):
        assert fn(f12, g) == O.zx_mul(fn(f1, g), fn(f2, g))


@pytest.mark.parametrize("seed", range(6))
def test_planted_common_factor_is_zero(seed):
    rng = random.Random(200 + seed)
    h = _rand_bipoly(rng, rng.randint(1, 2), 2)
    h[-1][0] = h[-1][0] or 1
    f = W._mul2(h, _rand_bipoly(rng, 2, 2))
    g = W._mul2(h, _rand_bipoly(rng, 2, 1))
    for fn in RES_METHODS.values():
        assert fn(f, g) == ()


def test_factor_in_x_only_does_not_vanish():
    """A common factor in Z[x] alone (deg_y = 0) does not make the resultant zero."""
    f = W._mul2([[1, 1]], [[1, 2], [3], [1]])
    g = W._mul2([[1, 1]], [[-1], [1, 1]])
    r = O.res_bareiss(f, g)
    assert r != ()
    assert O.res_subres(f, g) == r


# --------------------------------------------------------------------------- brute force


@pytest.mark.parametrize("seed", range(25))
def test_leibniz_brute_force(seed):
    """Tiny random inputs (degree <= 3, 2-bit coefficients), including zero leading
    coefficients in x, constant inputs and zero polynomials."""
    rng = random.Random(300 + seed)
    m, n = rng.randint(0, 3), rng.randint(0, 3)
    f = _rand_bipoly(rng, m, rng.randint(0, 2), -2, 1)
    g = _rand_bipoly(rng, n, rng.randint(0, 2), -2, 1)
    want = O.res_leibniz(f, g)
    assert O.res_bareiss(f, g) == want
    assert O.res_subres(f, g) == want
    assert O.res_evalz(f, g) == want


def test_degenerate_cases():
    f0 = [[3, 1]]            # m = 0: f = x + 3
    g = [[1, 2], [0, 1], [5]]   # n = 2
    assert O.res_bareiss(f0, g) == _zx_pow((3, 1), 2)
    assert O.res_subres(f0, g) == _zx_pow((3, 1), 2)
    assert O.res_bareiss(g, f0) == _zx_pow((3, 1), 2)      # n = 0 side, (-1)^(2*0) = 1
    assert O.res_bareiss([[2]], [[7, 1]]) == (1,)          # m = n = 0: empty determinant
    assert O.res_subres([[2]], [[7, 1]]) == (1,)
    assert O.res_bareiss([[0]], g) == ()                   # f = 0
    assert O.res_subres(g, [[0, 0]]) == ()
    assert O.res_evalz([[0]], g) == ()


def test_res_at_matches_polynomial_everywhere():
    """R(a) from the determinant at x = a equals the interpolated polynomial at a,
    including points where lc_y f or lc_y g vanishes (formal y-degrees kept)."""
    f = [[1, 2, -1], [0, 1], [-6, 1, 1]]      # lc_y f = x^2 + x - 6 = (x-2)(x+3)
    g = [[2, -1], [1, 0, 1], [-2, 1]]         # lc_y g = x - 2
    R = O.res_bareiss(f, g)
    for a in (-3, -1, 0, 1, 2, 3, 7):
        assert O.res_at(f, g, a) == O.zx_eval(R, a)
    assert O.res_evalz(f, g) == R


@pytest.mark.parametrize("seed", range(4))
def test_coefficients_within_hadamard_bound(seed):
    """|coeff| <= (sum_i ||f_i||_1^2)^(n/2) (sum_j ||g_j||_1^2)^(m/2) (Hadamard's
    inequality for the Sylvester matrix on |x| = 1)."""
    f, g = W.small_dense_pair(40 + seed, 5, 8)
    F, G = as_zxy(f), as_zxy(g)
    m, n = len(F) - 1, len(G) - 1
    sf = sum(sum(abs(c) for c in r) ** 2 for r in F)
    sg = sum(sum(abs(c) for c in r) ** 2 for r in G)
    R = O.res_subres(f, g)
    for c in R:
        assert c * c <= sf ** n * sg ** m


# --------------------------------------------------------------------------- the planned coefficient bound


def _log2_abs_interval(v: int):
    from oracle.bound import log2_interval

    return log2_interval(abs(v))


def _bound(f, g):
    from oracle.bound import resultant_bound_log2

    return resultant_bound_log2(f, g)


def test_bound_log2_interval_brackets():
    """The exact log2 enclosure against math.log2 (rationals, a + b sqrt 2)."""
    from fractions import Fraction

    from oracle.bound import log2_interval

    for x in (1, 2, 3, 5, 7, 1000, 2 ** 100 + 1, Fraction(1, 3), Fraction(7, 1024), Fraction(2 ** 90 - 1, 3 ** 40)):
        x = Fraction(x)
        lo, hi = log2_interval(x)
        v = math.log2(x.numerator) - math.log2(x.denominator)
        assert lo <= v + 1e-12 and v - 1e-12 <= hi and 0 < hi - lo < 1e-11
    for a, b in ((0, 1), (1, 1), (3, 2), (Fraction(1, 8), 5)):
        lo, hi = log2_interval(Fraction(a), Fraction(b))
        v = math.log2(a + b * math.sqrt(2))
        assert lo <= v + 1e-12 and v - 1e-12 <= hi
    # exact powers of two sit inside their enclosure
    for e in (0, 1, 17, 500, -30):
        lo, hi = log2_interval(Fraction(2) ** e)
        assert lo <= e <= hi


@pytest.mark.parametrize("a", [1, 3, 2 ** 20 + 7, 2 ** 40, 2 ** 200 - 5])
def test_bound_tight_two_by_two(a):
    """f = y + a, g = y - a: R = -2a, and the column form of the Hadamard bound is 2|a|
    for every lambda; f = y + a, g = a y - 1: R = -(1 + a^2), the row and column forms at
    lambda = 1.  The bound equals |R| (inside its enclosure)."""
    for f, g, r in (([[a], [1]], [[-a], [1]], 2 * a), ([[a], [1]], [[-1], [a]], 1 + a * a)):
        R = list(O.res_bareiss(f, g))
        assert R in ([-r], [r])
        lo, hi = _bound(f, g)
        l2lo, l2hi = _log2_abs_interval(r)
        assert lo <= l2hi and l2lo <= hi, (a, float(lo), float(hi))


@pytest.mark.parametrize("seed", range(6))
def test_bound_tight_constant_in_y(seed):
    """f = f_0(x) (y-degree 0) gives R = f_0^n, and |R(1)| = f_0(1)^n when f_0 has
    non-negative coefficients (|R(-1)| = |f_0(-1)|^n when they alternate): the bound
    n/2 log2 G(f_0) is then attained, so it equals log2 |R(+-1)| in both operand orders."""
    rng = random.Random(900 + seed)
    dx = rng.randint(0, 6)
    f0 = [rng.randint(0, 40) for _ in range(dx + 1)]
    f0[-1] = f0[-1] or 1
    alt = seed % 2 == 1
    if alt:
        f0 = [c if i % 2 == 0 else -c for i, c in enumerate(f0)]
    n = rng.randint(1, 4)
    g = [[rng.randint(-9, 9) for _ in range(rng.randint(1, 4))] for _ in range(n + 1)]
    g[-1][0] = g[-1][0] or 3
    x = -1 if alt else 1
    for A, B in (([f0], g), (g, [f0])):
        Rx = O.res_at(A, B, x)
        assert abs(Rx) == abs(sum(c * x ** i for i, c in enumerate(f0))) ** n
        lo, hi = _bound(A, B)
        l2lo, l2hi = _log2_abs_interval(Rx)
        assert lo <= l2hi and l2lo <= hi, (float(lo), float(hi), float(l2lo))


def _check_covers(f, g):
    R = O.res_subres(f, g)
    b = _bound(f, g)
    if not R:
        return
    assert b is not None
    vals = [max(abs(c) for c in R), abs(O.zx_eval(R, 1)), abs(O.zx_eval(R, -1))]
    for v in vals:
        if v:
            assert _log2_abs_interval(v)[0] <= b[1], (float(b[1]), v.bit_length())


@pytest.mark.parametrize("seed", range(12))
def test_bound_covers_resultants(seed):
    """max |coef R|, |R(1)| and |R(-1)| never exceed the bound: random dense pairs of
    mixed shapes (y-degree 0..5, x-degree 0..6, coefficients of 2..40 bits), pairs whose
    rows grow geometrically with the power of y (the best lambda is then not 1), and
    planted-roots pairs."""
    rng = random.Random(700 + seed)
    for _ in range(6):
        m, n = rng.randint(0, 5), rng.randint(0, 5)
        bits = rng.choice([2, 8, 20, 40])
        f = _rand_bipoly(rng, m, rng.randint(0, 6), -(1 << bits), 1 << bits)
        g = _rand_bipoly(rng, n, rng.randint(0, 6), -(1 << bits), 1 << bits)
        f[-1][0] = f[-1][0] or 1
        g[-1][0] = g[-1][0] or 1
        _check_covers(f, g)
    for s in (-12, -3, 5, 16):
        f = [[rng.randint(-9, 9) << max(0, s * i) for _ in range(3)] for i in range(4)]
        g = [[rng.randint(-9, 9) << max(0, -s * j) for _ in range(2)] for j in range(3)]
        f[-1][0] = f[-1][0] or 1
        g[-1][0] = g[-1][0] or 1
        _check_covers(f, g)
    f, g = W.planted_roots_pair(seed, 3, 2)[:2]
    _check_covers(f, g)


def test_summed_form_closed_forms():
    """The summed forms take the absolute values after summing the entries'
    autocorrelations.  h_0 = 1 + x and h_1 = 1 - x (A = [2, 1] and [2, -1]): at lambda = 1
    C_0 = 4 and C_1 = 0, so C_0 + 2|C_1| = 4 where the per-entry form gives 8; with the
    weights 1 and 2^(1/4) (lambda = 2^(1/8), degrees 0 and 1) C_0 = 2 + 2^(5/4) and
    C_1 = 1 - 2^(1/4), so C_0 + 2|C_1| = 2^(9/4)."""
    from fractions import Fraction

    from oracle import bound as B

    assert B.autocorr([1, 1]) == [2, 1] and B.autocorr([1, -1]) == [2, -1]
    for ents, q8, want in (([([2, 1], 0), ([2, -1], 0)], 0, Fraction(2)),
                           ([([2, 1], 0), ([2, -1], 1)], 1, Fraction(9, 4)),
                           ([([9, 2, -1], 2), ([1], 0)], 0, Fraction(4))):   # (9 + 1) + 2 (2 + 1) = 16
        lo, hi = B.summed_log2(ents, q8)
        assert lo <= want <= hi and hi - lo < Fraction(1, 2 ** 30), (ents, q8, float(lo), float(hi))
    assert B.autocorr_g([1, 1]) + B.autocorr_g([1, -1]) == 8


@pytest.mark.parametrize("seed", range(8))
def test_summed_forms_cover_and_tighten(seed):
    """On random pairs inside the summed forms' shapes (rows with cancelling
    autocorrelations among them) the bound with the summed forms still covers max |coef R|,
    |R(1)|, |R(-1)|, and it is never above the bound of the per-entry forms alone."""
    from oracle import bound as B

    rng = random.Random(1700 + seed)
    for _ in range(4):
        m, n = rng.randint(1, 5), rng.randint(1, 5)
        f = _rand_bipoly(rng, m, rng.randint(1, 6), -(1 << 12), 1 << 12)
        g = _rand_bipoly(rng, n, rng.randint(1, 6), -(1 << 12), 1 << 12)
        f[-1][0] = f[-1][0] or 1
        g[-1][0] = g[-1][0] or 1
        assert B.summed_eligible(f, g)
        _check_covers(f, g)
        both = B.hadamard_log2(f, g)
        old = B.hadamard_log2(f, g, summed=False)
        assert both[1] <= old[1]
    # a pair where they are strictly tighter: f = (1 + x) + (1 - x) y
    f, g = [[1, 1], [1, -1]], [[-3], [1]]
    assert B.hadamard_log2(f, g)[1] < B.hadamard_log2(f, g, summed=False)[0]
    _check_covers(f, g)


def test_bound_empty_column_and_degenerate():
    """A zero input gives no bound; constants in y give 0 = log2 1 for R = 1."""
    assert _bound([[0]], [[1], [2]]) is None
    assert _bound([[5]], [[7]]) == (0, 0)


# --------------------------------------------------------------------------- degree-6 workload


def test_small_dense_pair_methods_agree():
    f, g = W.small_dense_pair(1)
    r = O.res_bareiss(f, g)
    assert O.res_subres(f, g) == r
    assert O.res_evalz(f, g) == r
    assert len(r) - 1 <= 36
    for a in (-5, 0, 4, 99):
        assert O.res_at(f, g, a) == O.zx_eval(r, a)


# --------------------------------------------------------------------------- sympy cross-check


@pytest.mark.parametrize("seed", range(6))
def test_sympy_resultant(seed):
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    rng = random.Random(400 + seed)
    f = _rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 3), -9, 9)
    g = _rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 3), -9, 9)
    f[-1][-1] = f[-1][-1] or 1
    g[-1][-1] = g[-1][-1] or 1
    F = sum(c * x ** i * y ** j for j, r in enumerate(f) for i, c in enumerate(r))
    G = sum(c * x ** i * y ** j for j, r in enumerate(g) for i, c in enumerate(r))
    s = sympy.Poly(sympy.resultant(F, G, y), x)
    want = O.zx_trim(int(c) for c in reversed(s.all_coeffs()))
    assert O.res_subres(f, g) == want
    assert O.res_bareiss(f, g) == want


@pytest.mark.parametrize("seed", range(6))
def test_sympy_gcd(seed):
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    rng = random.Random(500 + seed)
    h = [rng.randint(-5, 5) for _ in range(rng.randint(1, 4))]
    h[-1] = h[-1] or 3
    p = O.zx_mul(tuple(h), tuple(rng.randint(-9, 9) for _ in range(rng.randint(1, 6))))
    q = O.zx_mul(tuple(h), tuple(rng.randint(-9, 9) for _ in range(rng.randint(1, 6))))
    s = sympy.Poly(sympy.gcd(sympy.Poly(list(reversed(p)) or [0], x), sympy.Poly(list(reversed(q)) or [0], x)), x)
    want = O.zx_trim(int(c) for c in reversed(s.all_coeffs()))
    if want and want[-1] < 0:
        want = O.zx_neg(want)
    assert O.gcd_z(p, q) == want


# --------------------------------------------------------------------------- gcd invariants


@pytest.mark.parametrize("seed", range(6))
def test_gcd_planted_factor_and_cofactors(seed):
    P, Q, H = W.gcd_batch(seed + 10, 1, lo=8, hi=20, hdeg=3)
    p, q, h = P[0], Q[0], H[0]
    G = O.gcd_z(p, q)
    assert G and G[-1] > 0
    assert O.divides_z(G, p) and O.divides_z(G, q)
    assert O.divides_z(h, G)                        # the planted factor divides the gcd
    cp, cq = O.zx_divexact(O.zx_trim(p), G), O.zx_divexact(O.zx_trim(q), G)
    assert O.res_univariate(list(cp), list(cq), O.ZZ) != 0   # cofactors coprime
    assert O.content(cp) and math.gcd(O.content(cp), O.content(cq)) == 1


def test_gcd_content_multiplies():
    p = O.zx_mul((6,), O.zx_mul((1, 1), (2, 0, 1)))      # 6 (x+1)(x^2+2)
    q = O.zx_mul((4,), O.zx_mul((1, 1), (3, 1)))          # 4 (x+1)(x+3)
    assert O.gcd_z(p, q) == (2, 2)
    assert O.gcd_z(O.zx_neg(p), q) == (2, 2)


def test_gcd_coprime_is_content_gcd():
    assert O.gcd_z((3, 6, 9), (6, 0, 12, 6)) == (3,)
    assert O.gcd_z((1, 1), (1, -1)) == (1,)


@pytest.mark.parametrize("seed", range(6))
def test_subres_abnormal_sequences(seed):
    """Polynomials with gaps in their y-support give remainder sequences whose degrees
    drop by two or more after the first step (delta >= 2 with h != 1), the one branch
    of the subresultant recurrence the dense inputs never reach."""
    rng = random.Random(600 + seed)
    f = [[0]] * 7
    g = [[0]] * 6
    f = [list(r) for r in f]
    g = [list(r) for r in g]
    f[6] = [rng.choice([1, 2, -3])]
    f[3] = [rng.randint(-4, 4), rng.randint(-4, 4)]
    f[0] = [rng.randint(-4, 4), 1]
    g[5] = [rng.choice([1, -1, 2])]
    g[2] = [rng.randint(-4, 4), rng.randint(-2, 2)]
    g[0] = [rng.randint(-4, 4)]
    want = O.res_bareiss(f, g)
    assert O.res_subres(f, g) == want
    assert O.res_evalz(f, g) == want
    for a in (-2, 0, 3):
        Fa = [O.zx_eval(O.zx_trim(r), a) for r in f]
        Ga = [O.zx_eval(O.zx_trim(r), a) for r in g]
        assert O.res_univariate(Fa, Ga, O.ZZ) == O.zx_eval(want, a)


def test_res_at_prs_matches_determinant():
    f, g = W.small_dense_pair(7, 4, 8)
    for a in (-9, 0, 5, 123456):
        assert O.res_at_prs(f, g, a) == O.res_at(f, g, a)
    fl = [[1, 2, -1], [0, 1], [-6, 1, 1]]       # lc vanishes at 2 and -3
    gl = [[2, -1], [1, 0, 1], [-2, 1]]
    for a in (-3, 2, 4):
        assert O.res_at_prs(fl, gl, a) == O.res_at(fl, gl, a)


# --------------------------------------------------------------------------- square-free factorisation


def _planted_sqf(rng, mults, nroots=3, lc_choices=(1, 2, 3, 5)):
    """u * prod r_i^i with every r_i a product of distinct primitive linear factors
    (b x - a), gcd(a, b) = 1, all ratios a / b distinct: square-free, pairwise coprime
    and primitive by construction."""
    used = set()
    factors = []
    for _ in range(mults):
        r = (1,)
        for _ in range(rng.randint(0, nroots)):
            while True:
                b = rng.choice(lc_choices)
                a = rng.randint(-9, 9)
                if math.gcd(a, b) == 1 and (a, b) not in used and all(a * bb != aa * b for aa, bb in used):
                    break
            used.add((a, b))
            r = O.zx_mul(r, (-a, b))
        factors.append(r)
    while factors and len(factors[-1]) == 1:
        factors.pop()
    u = rng.choice([1, -1, 6, -10, 35])
    R = (u,)
    for i, r in enumerate(factors, start=1):
        R = O.zx_mul(R, _zx_pow(r, i))
    return u, factors, R


@pytest.mark.parametrize("seed", range(12))
def test_sqf_planted_factorisation(seed):
    rng = random.Random(900 + seed)
    u, factors, R = _planted_sqf(rng, rng.randint(1, 4))
    assert O.sqf_yun(R) == (u, factors)


def test_sqf_hand_cases():
    assert O.sqf_yun([]) == (0, [])
    assert O.sqf_yun([-6]) == (-6, [])
    assert O.sqf_yun([-3, 6, -3]) == (-3, [(1,), (-1, 1)])           # -3 (x - 1)^2
    assert O.sqf_yun([0, 0, 0, 4]) == (4, [(1,), (1,), (0, 1)])      # 4 x^3
    assert O.sqf_yun([-2, 0, 2]) == (2, [(-1, 0, 1)])                 # 2 (x^2 - 1)


@pytest.mark.parametrize("seed", range(6))
def test_sqf_against_sympy(seed):
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    rng = random.Random(950 + seed)
    R = (rng.choice([1, -2, 3]),)
    for _ in range(rng.randint(1, 4)):
        p = tuple(rng.randint(-5, 5) for _ in range(rng.randint(2, 4)))
        R = O.zx_mul(R, _zx_pow(O.zx_trim(p) or (1,), rng.randint(1, 3)))
    u, facs = O.sqf_yun(R)
    coeff, lst = sympy.sqf_list(sympy.Poly(list(reversed(R)), x))
    mult = {}
    for fac, e in lst:
        c = fac.all_coeffs()
        if c[0] < 0:
            c = [-v for v in c]
            coeff = -coeff
        mult[e] = tuple(int(v) for v in reversed(c))
    want = [mult.get(i, (1,)) for i in range(1, (max(mult) if mult else 0) + 1)]
    assert facs == want and u == int(coeff)


@pytest.mark.parametrize("seed", range(4))
def test_sqf_invariants_on_discriminant_resultant(seed):
    """R = res_y(f, f_y) of a union of two circles (singular where they meet): u prod r_i^i equals R,
    every r_i is primitive with positive leading coefficient and the r_i are pairwise
    coprime (checked with sympy's gcd where available, by trial division otherwise)."""
    rng = random.Random(970 + seed)

    def circle(a, b, r):   # (x - a)^2 + (y - b)^2 - r^2, rows = powers of y
        return [[a * a + b * b - r * r, -2 * a, 1], [-2 * b], [1]]

    # two circles: a square-free curve, singular where they meet (repeated roots of R)
    f = W._mul2(circle(rng.randint(-3, 3), rng.randint(-3, 3), rng.randint(2, 4)),
                circle(rng.randint(-3, 3), rng.randint(-3, 3), rng.randint(2, 4)))
    R = O.disc_res(f)
    assert O.zx_trim(R)
    u, facs = O.sqf_yun(R)
    prod = (u,)
    for i, r in enumerate(facs, start=1):
        assert r[-1] > 0 and O.content(r) == 1
        prod = O.zx_mul(prod, _zx_pow(r, i))
    assert prod == O.zx_trim(R)
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    polys = [sympy.Poly(list(reversed(r)), x) for r in facs]
    for i in range(len(polys)):
        assert sympy.degree(sympy.gcd(polys[i], polys[i].diff(x)), x) <= 0
        for j in range(i):
            assert sympy.degree(sympy.gcd(polys[i], polys[j]), x) <= 0


# --------------------------------------------------------------------------- bivariate gcd, Teissier Q

def _rows_mul(a, b):
    out = [[0] * (max(len(r) for r in a) + max(len(r) for r in b) - 1) for _ in range(len(a) + len(b) - 1)]
    for j1, r1 in enumerate(a):
        for i1, c1 in enumerate(r1):
            if c1:
                for j2, r2 in enumerate(b):
                    for i2, c2 in enumerate(r2):
                        out[j1 + j2][i1 + i2] += c1 * c2
    return out


def _rand_bivariate(rng, dy, dx, amp):
    f = [[rng.randint(-amp, amp) for _ in range(dx + 1)] for _ in range(dy + 1)]
    f[dy][rng.randint(0, dx)] = rng.choice([1, -1, 2, 3])
    return f


def test_bigcd_hand_cases():
    from oracle.bigcd import content_y, gcd_zxy, teissier_parts, teissier_q

    xpy, xmy = [[0, 1], [1]], [[0, 1], [-1]]
    assert gcd_zxy([[0, 0], [0, 1]], [[0, 0, 1]]) == [(0, 1)]                 # gcd(x y, x^2) = x
    assert gcd_zxy(_rows_mul(xpy, xpy), _rows_mul(xpy, xmy)) == [(0, 1), (1,)]   # x + y
    assert gcd_zxy([[0]], [[0]]) == []
    assert gcd_zxy([[0, 0], [0, -3]], [[0]]) == [(), (0, 3)]                 # gcd(-3 x y, 0) = 3 x y
    assert content_y([[4, 2], [0, 2]]) == (2,)                               # 2 x y + 2 x + 4
    assert content_y([[0, 2], [0, 4]]) == (0, 2)                             # 4 x y + 2 x
    f = _rows_mul(xpy, xpy)
    f[0][0] += 1                                                             # (x + y)^2 + 1
    h, fxs, fys = teissier_parts(f)
    assert h == [(0, 2), (2,)] and fxs == [(1,)] and fys == [(1,)] and teissier_q(f) == (1,)


@pytest.mark.parametrize("seed", range(10))
def test_bigcd_planted_factor(seed):
    """A planted common factor h divides the gcd, the gcd divides both inputs, and
    the cofactors are coprime: their contents have gcd 1 (gcd_z) and at some
    integer x = a with non-vanishing leading coefficients their univariate gcd in y
    is constant."""
    from oracle.bigcd import content_y, divexact_zxy, gcd_zxy

    rng = random.Random(4100 + seed)
    h = _rand_bivariate(rng, rng.randint(1, 2), rng.randint(0, 2), 3)
    u = _rand_bivariate(rng, rng.randint(0, 2), rng.randint(0, 2), 5)
    v = _rand_bivariate(rng, rng.randint(0, 2), rng.randint(0, 2), 5)
    if seed % 3 == 0:                       # a shared factor in x alone as well
        u = _rows_mul(u, [[seed + 1, 1]])
        v = _rows_mul(v, [[seed + 1, 1]])
    f, g = _rows_mul(h, u), _rows_mul(h, v)
    G = gcd_zxy(f, g)
    assert divexact_zxy(G, [tuple(r) for r in O.bigcd.as_zxy(h)]) is not None      # h | G
    a, b = divexact_zxy(f, G), divexact_zxy(g, G)                            # G | f, G | g
    assert O.gcd_z(content_y(a), content_y(b)) == (1,)
    ok = False
    for x0 in range(-6, 7):
        ra = [O.zx_eval(r, x0) for r in a]
        rb = [O.zx_eval(r, x0) for r in b]
        if ra[-1] == 0 or rb[-1] == 0:
            continue
        if len(O.gcd_z(ra, rb)) == 1:
            ok = True
            break
    assert ok
    assert G[-1][-1] > 0


@pytest.mark.parametrize("seed", range(6))
def test_bigcd_against_sympy(seed):
    sympy = pytest.importorskip("sympy")
    from oracle.bigcd import gcd_zxy

    x, y = sympy.symbols("x y")
    rng = random.Random(4200 + seed)
    h = _rand_bivariate(rng, rng.randint(0, 2), rng.randint(0, 2), 4)
    u = _rand_bivariate(rng, rng.randint(0, 2), rng.randint(0, 3), 6)
    v = _rand_bivariate(rng, rng.randint(0, 2), rng.randint(0, 3), 6)
    f, g = _rows_mul(h, u), _rows_mul(h, v)

    def expr(rows):
        return sum(c * x**i * y**j for j, r in enumerate(rows) for i, c in enumerate(r))

    want = sympy.Poly(sympy.gcd(expr(f), expr(g)), y, x)
    got = sympy.Poly(expr([list(r) for r in gcd_zxy(f, g)]), y, x)
    assert got == want or got == -want


@pytest.mark.parametrize("seed", range(4))
def test_teissier_q_against_sympy(seed):
    sympy = pytest.importorskip("sympy")
    from oracle.bigcd import teissier_q

    x, y = sympy.symbols("x y")
    rng = random.Random(4300 + seed)
    if seed % 2 == 0:                       # f = g(x + 2y) + (small perturbation in x only)
        L = [[0, 1], [2]]
        f, p = [[rng.randint(-4, 4)]], [[1]]
        for k in range(1, 4):
            p = _rows_mul(p, L)
            c = rng.randint(-3, 3) or 1
            f = [[(f[j][i] if j < len(f) and i < len(f[j]) else 0) + c * (p[j][i] if j < len(p) and i < len(p[j]) else 0)
                  for i in range(max(len(r) for r in f + p))] for j in range(max(len(f), len(p)))]
    else:                                   # a generic curve: gcd(f_x, f_y) = 1
        f = _rand_bivariate(rng, 3, 3, 5)

    def expr(rows):
        return sum(c * x**i * y**j for j, r in enumerate(rows) for i, c in enumerate(r))

    F = expr(f)
    fx, fy = sympy.diff(F, x), sympy.diff(F, y)
    h = sympy.gcd(fx, fy)
    Q = sympy.resultant(sympy.quo(fx, h), sympy.quo(fy, h), y)
    want = sympy.Poly(Q, x).all_coeffs()[::-1] if Q != 0 else []
    got = list(teissier_q(f))
    while want and want[-1] == 0:
        want.pop()
    assert got == [int(c) for c in want] or got == [-int(c) for c in want]


def test_teissier_q_degenerate_curves():
    """Q = res(f_x/h, f_y/h, y) is the zero polynomial () when f_x or f_y vanishes
    (Section 2.1 with the determinant convention res(0, g) = 0): a curve in y
    alone (f_x = 0, h = f_y up to its sign), in x alone (f_y = 0) and a constant
    (h = gcd(0, 0) = 0)."""
    from oracle.bigcd import teissier_parts, teissier_q

    fy_only = [[1], [0], [1]]                                   # y^2 + 1
    h, fxs, fys = teissier_parts(fy_only)
    assert h == [(), (2,)] and fxs == [] and fys == [(1,)]      # h = 2y, f_x / h = 0, f_y / h = 1
    assert teissier_q(fy_only) == ()
    fx_only = [[5, -1, 0, 1]]                                   # x^3 - x + 5
    h, fxs, fys = teissier_parts(fx_only)
    assert h == [(-1, 0, 3)] and fxs == [(1,)] and fys == []
    assert teissier_q(fx_only) == ()
    assert teissier_parts([[7]]) == ([], [], []) and teissier_q([[7]]) == ()


def test_teissier_q_generic_curve_is_the_plain_resultant():
    """gcd(f_x, f_y) = 1 for a generic curve, so Q = res(f_x, f_y) itself (with the
    x-derivative taken row by row)."""
    from oracle.bigcd import deriv_x, teissier_parts, teissier_q

    rng = random.Random(4400)
    f = _rand_bivariate(rng, 4, 4, 9)
    h, _, _ = teissier_parts(f)
    assert len(h) == 1 and len(h[0]) == 1                        # a constant
    fx = [list(r) or [0] for r in deriv_x(f)]
    fy = [list(r) or [0] for r in O.deriv_y(f)]
    want = O.res_subres(fx, fy)
    c = h[0][0]
    # res(f_x / c, f_y / c) = c^-(deg f_x + deg f_y) res(f_x, f_y) in y
    m, n = O.ydeg(fx), O.ydeg(fy)
    assert tuple(v * c ** (m + n) for v in teissier_q(f)) == tuple(want)
