"""Exact resultants over Z[x] (test infrastructure only).

Definition followed (Section 2.1 "Projection Phase", Section 3 "Arrangement
Computation"): for f, g in Z[x][y] with y-degrees m and n taken over Z[x]
(leading coefficients are non-zero polynomials in x),

    res_y(f, g) = det Syl_y(f, g),

the (m+n) x (m+n) Sylvester matrix whose first n rows hold the coefficients of
f and whose last m rows hold those of g, in decreasing powers of y, each row
shifted one column to the right of the one above.  With this orientation
res(g, f) = (-1)^(m n) res(f, g) and, for f = a prod (y - alpha_i),
g = b prod (y - beta_j), res(f, g) = a^n b^m prod (alpha_i - beta_j).

Degenerate cases follow the determinant: f = 0 or g = 0 gives 0; m = 0 gives
f_0^n; n = 0 gives g_0^m; m = n = 0 gives 1 (empty determinant).
"""

from __future__ import annotations

import itertools
from fractions import Fraction  # noqa: F401  (kept for readers checking exactness by hand)

from .zpoly import ZX, ZZ, zx_eval, zx_trim, zx_mul, zx_add


# --------------------------------------------------------------------------- input helpers


def as_zxy(f) -> list[tuple]:
    """Bivariate input (rows f[j][i] = coeff of x^i y^j, list or array) -> list over y of
    Z[x] tuples, with zero rows above the y-degree removed."""
    rows = [zx_trim(int(c) for c in row) for row in f]
    while rows and not rows[-1]:
        rows.pop()
    return rows


def ydeg(f) -> int:
    return len(as_zxy(f)) - 1


def xdeg(f) -> int:
    return max((len(r) - 1 for r in as_zxy(f)), default=-1)


def deriv_y(f) -> list[list[int]]:
    """df/dy as rows: row j of the result is (j+1) * row (j+1) of f."""
    F = [list(int(c) for c in row) for row in f]
    if len(F) <= 1:
        return [[0]]
    return [[(j + 1) * c for c in F[j + 1]] for j in range(len(F) - 1)]


def degree_bound(F: list[tuple], G: list[tuple]) -> int:
    """deg_x res_y(f, g) <= n * deg_x f + m * deg_x g: every term of the Leibniz
    expansion takes n entries from the f rows and m from the g rows."""
    m, n = len(F) - 1, len(G) - 1
    dxf = max(len(r) - 1 for r in F)
    dxg = max(len(r) - 1 for r in G)
    return max(0, n * dxf + m * dxg)


# --------------------------------------------------------------------------- determinants


def sylvester(F: list, G: list, ring) -> list[list]:
    """Sylvester matrix of F (formal degree len(F)-1) and G (formal degree len(G)-1);
    F, G are coefficient lists over `ring`, lowest power of y first."""
    m, n = len(F) - 1, len(G) - 1
    N = m + n
    M = [[ring.zero] * N for _ in range(N)]
    for r in range(n):                      # n rows of f
        for t in range(m + 1):
            M[r][r + t] = F[m - t]
    for r in range(m):                      # m rows of g
        for t in range(n + 1):
            M[n + r][r + t] = G[n - t]
    return M


def det_bareiss(M: list[list], ring):
    """Fraction-free Gaussian elimination (Bareiss): after step k every entry of the
    trailing block is a (k+1)-minor, so the division by the previous pivot is exact.
    A zero pivot is replaced by a row swap, which flips the sign."""
    n = len(M)
    if n == 0:
        return ring.one
    A = [list(row) for row in M]
    sign = 1
    prev = ring.one
    for k in range(n - 1):
        if ring.is_zero(A[k][k]):
            piv = next((i for i in range(k + 1, n) if not ring.is_zero(A[i][k])), None)
            if piv is None:
                return ring.zero
            A[k], A[piv] = A[piv], A[k]
            sign = -sign
        akk = A[k][k]
        for i in range(k + 1, n):
            aik = A[i][k]
            for j in range(k + 1, n):
                A[i][j] = ring.divexact(ring.sub(ring.mul(A[i][j], akk), ring.mul(aik, A[k][j])), prev)
        prev = akk
    d = A[n - 1][n - 1]
    return d if sign > 0 else ring.neg(d)


def _perm_sign(p) -> int:
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def det_leibniz(M: list[list], ring):
    """Sum over all permutations (brute force; only for matrices up to about 8 x 8)."""
    n = len(M)
    total = ring.zero
    for p in itertools.permutations(range(n)):
        term = ring.one
        for i in range(n):
            term = ring.mul(term, M[i][p[i]])
            if ring.is_zero(term):
                break
        if ring.is_zero(term):
            continue
        total = ring.add(total, term) if _perm_sign(p) > 0 else ring.sub(total, term)
    return total


def _zero_or_swap(F, G):
    if not F or not G:
        return True
    return False


def res_bareiss(f, g) -> tuple:
    """res_y(f, g) in Z[x] as the Bareiss determinant of the Sylvester matrix over Z[x]."""
    F, G = as_zxy(f), as_zxy(g)
    if _zero_or_swap(F, G):
        return ()
    return det_bareiss(sylvester(F, G, ZX), ZX)


def res_leibniz(f, g) -> tuple:
    """res_y(f, g) by permutation expansion of the Sylvester determinant (tiny inputs)."""
    F, G = as_zxy(f), as_zxy(g)
    if _zero_or_swap(F, G):
        return ()
    return det_leibniz(sylvester(F, G, ZX), ZX)


# --------------------------------------------------------------------------- subresultant PRS


def _prem(A: list, B: list, ring) -> list:
    """Pseudo-remainder: lc(B)^(deg A - deg B + 1) * A mod B (exactly that power)."""
    r = list(A)
    db = len(B) - 1
    lb = B[db]
    for k in range(len(A) - 1, db - 1, -1):
        c = r[k]
        r = [ring.mul(lb, x) for x in r]
        if not ring.is_zero(c):
            for t in range(db + 1):
                r[k - db + t] = ring.sub(r[k - db + t], ring.mul(c, B[t]))
    r = r[:db]
    while r and ring.is_zero(r[-1]):
        r.pop()
    return r


def _pow(a, e: int, ring):
    out = ring.one
    for _ in range(e):
        out = ring.mul(out, a)
    return out


def res_univariate(A: list, B: list, ring):
    """res(A, B) for coefficient lists over an integral domain with non-zero leading
    coefficients, by the subresultant remainder sequence (Collins; Brown-Traub).

    Each pseudo-remainder is divided by g * h^delta, which the subresultant theorem
    shows to be exact; g tracks the leading coefficient of the current divisor and h
    the leading coefficient of the last subresultant.  The result is
    s * lc(last)^deg / h^(deg-1) where s collects the sign changes
    (-1)^(deg A deg B) of the swaps."""
    if not A or not B:
        return ring.zero
    da, db = len(A) - 1, len(B) - 1
    s = 1
    if da < db:
        A, B = B, A
        da, db = db, da
        if (da * db) % 2:
            s = -s
    if db == 0:
        v = _pow(B[0], da, ring)
        return v if s > 0 else ring.neg(v)
    g = ring.one
    h = ring.one
    while True:
        delta = da - db
        if da % 2 and db % 2:
            s = -s
        R = _prem(A, B, ring)
        A, da = B, db
        if not R:
            return ring.zero
        div = ring.mul(g, _pow(h, delta, ring))
        B = [ring.divexact(c, div) for c in R]
        db = len(B) - 1
        g = A[da]
        if delta == 0:
            pass
        else:
            h = ring.divexact(_pow(g, delta, ring), _pow(h, delta - 1, ring))
        if db == 0:
            v = ring.divexact(_pow(B[0], da, ring), _pow(h, da - 1, ring)) if da >= 1 else ring.one
            return v if s > 0 else ring.neg(v)


def res_subres(f, g) -> tuple:
    """res_y(f, g) in Z[x] by the subresultant remainder sequence over Z[x][y]."""
    F, G = as_zxy(f), as_zxy(g)
    if _zero_or_swap(F, G):
        return ()
    return res_univariate(F, G, ZX)


# --------------------------------------------------------------------------- evaluation over Z


def res_at(f, g, a: int) -> int:
    """R(a) for R = res_y(f, g): the Sylvester determinant at x = a, keeping the
    y-degrees of f and g over Z[x] even where their leading coefficients vanish at a."""
    F, G = as_zxy(f), as_zxy(g)
    if _zero_or_swap(F, G):
        return 0
    Fa = [zx_eval(c, a) for c in F]
    Ga = [zx_eval(c, a) for c in G]
    return det_bareiss(sylvester(Fa, Ga, ZZ), ZZ)


def res_evalz(f, g) -> tuple:
    """res_y(f, g) by exact evaluation and interpolation over Z (no primes).

    The window of D+1 consecutive integers a0, a0+1, ... (D = n deg_x f + m deg_x g)
    is chosen to avoid the integer roots of lc_y(f) lc_y(g), so both y-degrees are
    kept at every point and the integer resultant per point is the subresultant one.
    Newton's divided differences on a unit-spaced grid are Delta^j v / j!, which are
    integers for an integer polynomial; the division is asserted exact."""
    F, G = as_zxy(f), as_zxy(g)
    if _zero_or_swap(F, G):
        return ()
    D = degree_bound(F, G)
    lf, lg = F[-1], G[-1]
    a0 = 0
    while any(zx_eval(lf, a) * zx_eval(lg, a) == 0 for a in range(a0, a0 + D + 1)):
        a0 += 1
    vals = []
    for t in range(D + 1):
        a = a0 + t
        vals.append(res_univariate([zx_eval(c, a) for c in F], [zx_eval(c, a) for c in G], ZZ))
    return _interp_unit_grid(vals, a0)


def _interp_unit_grid(vals: list[int], a0: int) -> tuple:
    D = len(vals) - 1
    d = list(vals)
    newton = [d[0]]
    fact = 1
    for j in range(1, D + 1):
        d = [d[i + 1] - d[i] for i in range(len(d) - 1)]
        fact *= j
        q, r = divmod(d[0], fact)
        if r:
            raise ArithmeticError("non-integral Newton coefficient")
        newton.append(q)
    poly: tuple = ()
    for j in range(D, -1, -1):
        poly = zx_add(zx_mul(poly, (-(a0 + j), 1)), (newton[j],))
    return poly


def disc_res(f, method: str = "subres") -> tuple:
    """res_y(f, df/dy) in Z[x] (Section 2.1), not divided by the leading coefficient."""
    fy = deriv_y(f)
    fn = {"subres": res_subres, "bareiss": res_bareiss, "evalz": res_evalz}[method]
    return fn(f, fy)


def res_at_prs(f, g, a: int) -> int:
    """R(a) by the integer subresultant sequence when lc_y f(a) lc_y g(a) != 0 (both
    y-degrees kept), else by the Sylvester determinant (res_at)."""
    F, G = as_zxy(f), as_zxy(g)
    if _zero_or_swap(F, G):
        return 0
    if zx_eval(F[-1], a) == 0 or zx_eval(G[-1], a) == 0:
        return res_at(f, g, a)
    return res_univariate([zx_eval(c, a) for c in F], [zx_eval(c, a) for c in G], ZZ)
