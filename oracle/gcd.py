"""Exact gcd in Z[x] (test infrastructure only).

Definition followed (Section 2, Algorithm: content removal h = gcd(f_0, f_1, ...);
Section 2.1: square-free factorisation by gcds): the greatest common divisor of
two integer polynomials, normalised to a positive leading coefficient, including
the gcd of their integer contents.  gcd(0, 0) = 0 and gcd(p, 0) = p / sign(lc p).

Method: the primitive polynomial remainder sequence over Z - repeated
pseudo-division followed by removal of the integer content - whose last non-zero
member is the primitive part of the gcd.
"""

from __future__ import annotations

import math

from .zpoly import zx_trim, content, primitive_part, zx_divexact


def _prem(a: list[int], b: list[int]) -> list[int]:
    r = list(a)
    db = len(b) - 1
    lb = b[db]
    for k in range(len(a) - 1, db - 1, -1):
        c = r[k]
        r = [lb * x for x in r]
        if c:
            for t in range(db + 1):
                r[k - db + t] -= c * b[t]
    return list(zx_trim(r[:db]))


def gcd_z(p, q) -> tuple:
    """gcd(p, q) in Z[x] with positive leading coefficient."""
    p = zx_trim(int(c) for c in p)
    q = zx_trim(int(c) for c in q)
    if not p and not q:
        return ()
    if not q:
        return tuple(-c for c in p) if p[-1] < 0 else p
    if not p:
        return tuple(-c for c in q) if q[-1] < 0 else q
    c = math.gcd(content(p), content(q))
    a, b = list(primitive_part(p)), list(primitive_part(q))
    if len(a) < len(b):
        a, b = b, a
    while b:
        r = _prem(a, b)
        a, b = b, (list(primitive_part(r)) if r else [])
    g = primitive_part(a)
    return tuple(c * x for x in g)


def divides_z(d, p) -> bool:
    """True when d divides p in Z[x]."""
    try:
        zx_divexact(zx_trim(p), zx_trim(d))
        return True
    except ArithmeticError:
        return False
