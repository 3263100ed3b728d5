"""Bivariate gcd in Z[x][y], content removal and the Teissier resultant Q
(test infrastructure only).

Definitions followed:
* Section 2 (Algorithm, content removal): the content of f with respect to y is
  h = gcd(f_0, f_1, ...) in Z[x] of its y-coefficients; dividing it out removes
  vertical components.
* Section 2.1 (the Teissier bound): for a curve f, h = gcd(f_x, f_y) in Z[x, y],
  f_x* = f_x / h, f_y* = f_y / h and Q = res(f_x*, f_y*, y) in Z[x]; the number of
  distinct roots of f(alpha, y) is at most deg_y f - mult(R, alpha) + mult(Q, alpha).

Readings: the gcd in Z[x][y] is unique up to sign; it is normalised so that the
leading coefficient (in x) of its leading coefficient in y is positive, and it
includes the gcd of the arguments' contents (as gcd_z does for Z[x]).  gcd(0, 0) = 0.

Method (Gauss's lemma, one variable at a time): the content in Z[x] of each
argument (gcd_z of its y-coefficients), the primitive parts, and the primitive
remainder sequence over Z[x] - pseudo-division in y followed by removal of the
Z[x]-content - whose last non-zero member is the primitive part of the gcd.

Bivariate polynomials are lists of rows, row j the Z[x] tuple of y^j (lowest
powers first), the layout of the resultant oracle.
"""

from __future__ import annotations

from .gcd import gcd_z
from .resultant import _prem, as_zxy, res_subres
from .zpoly import ZX, zx_divexact, zx_mul, zx_sub, zx_trim


def _trim_rows(rows) -> list:
    rows = [zx_trim(r) for r in rows]
    while rows and not rows[-1]:
        rows.pop()
    return rows


def content_y(f) -> tuple:
    """gcd in Z[x] of the y-coefficients of f (positive leading coefficient); () for 0."""
    g = ()
    for row in as_zxy(f):
        g = gcd_z(g, row)
    return g


def pp_y(f) -> list:
    """f divided by its content with respect to y (rows); [] for 0."""
    F = as_zxy(f)
    c = content_y(F)
    return [zx_divexact(r, c) if r else () for r in F] if c else []


def divexact_zxy(a, b) -> list:
    """a / b in Z[x][y] by long division in y with exact divisions in Z[x];
    ArithmeticError when b does not divide a."""
    A, B = _trim_rows(as_zxy(a)), _trim_rows(as_zxy(b))
    if not B:
        raise ZeroDivisionError("division by the zero polynomial")
    db = len(B) - 1
    Q = [()] * max(len(A) - db, 0)
    while A and len(A) - 1 >= db:
        k = len(A) - 1 - db
        q = zx_divexact(A[-1], B[-1])
        Q[k] = q
        for t in range(db + 1):
            A[k + t] = zx_sub(A[k + t], zx_mul(q, B[t]))
        A = _trim_rows(A)
    if A:
        raise ArithmeticError("not an exact division in Z[x][y]")
    return _trim_rows(Q)


def _normalise(rows) -> list:
    if rows and rows[-1][-1] < 0:
        return [tuple(-c for c in r) for r in rows]
    return rows


def gcd_zxy(f, g) -> list:
    """gcd(f, g) in Z[x][y], normalised as described in the module docstring."""
    F, G = _trim_rows(as_zxy(f)), _trim_rows(as_zxy(g))
    if not F and not G:
        return []
    if not G:
        return _normalise(F)
    if not F:
        return _normalise(G)
    c = gcd_z(content_y(F), content_y(G))
    A, B = pp_y(F), pp_y(G)
    if len(A) < len(B):
        A, B = B, A
    while B:
        r = _prem(list(A), list(B), ZX)
        A, B = B, (pp_y(r) if r else [])
    H = pp_y(A)
    return _normalise([zx_mul(c, row) for row in H])


def deriv_x(f) -> list:
    """df/dx as rows."""
    return [tuple(i * row[i] for i in range(1, len(row))) for row in as_zxy(f)] or [()]


def deriv_yx(f) -> list:
    """df/dy as rows."""
    F = as_zxy(f)
    return [tuple((j + 1) * c for c in F[j + 1]) for j in range(len(F) - 1)] or [()]


def teissier_parts(f) -> tuple:
    """(h, f_x*, f_y*) with h = gcd(f_x, f_y) in Z[x, y] and f_x* = f_x / h,
    f_y* = f_y / h (Section 2.1)."""
    fx, fy = _trim_rows(deriv_x(f)), _trim_rows(deriv_yx(f))
    h = gcd_zxy(fx, fy)
    if not h:
        return [], fx, fy
    return h, divexact_zxy(fx, h), divexact_zxy(fy, h)


def teissier_q(f) -> tuple:
    """Q = res(f_x*, f_y*, y) in Z[x] (Section 2.1), by the subresultant PRS."""
    _, fxs, fys = teissier_parts(f)
    if not fxs or not fys:
        return ()
    return res_subres([list(r) or [0] for r in fxs], [list(r) or [0] for r in fys])
