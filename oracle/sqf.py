"""Square-free factorisation in Z[x] (test infrastructure only).

Definition followed (Section 2.1, Projection Phase): R = prod_i r_i^i with
square-free, pairwise coprime r_i in Z[x] (r_i = 1 for multiplicities that do
not occur), obtained by Yun's algorithm - gcds of R and its derivative, then of
the successive quotients.  Reading for Z[x]: R = u * prod_i r_i^i with every r_i
primitive with a positive leading coefficient and u an integer (the content of
R with the sign of its leading coefficient).

Method (Yun, over Z with primitive gcds, in the order of the algorithm):
  A = R / u (primitive, lc > 0), B = A'
  G = gcd(A, B), C = A / G, D = B / G - C'
  repeat: r_i = gcd(C, D); C = C / r_i; D = D / r_i - C'   until deg C = 0
Every division is exact in Z[x] (Gauss's lemma: the divisors are primitive).
"""

from __future__ import annotations

from .gcd import gcd_z
from .zpoly import content, zx_divexact, zx_sub, zx_trim


def _deriv(a) -> tuple:
    return zx_trim(i * a[i] for i in range(1, len(a)))


def sqf_yun(r) -> tuple[int, list[tuple]]:
    """(u, [r_1, ..., r_m]) with R = u * prod r_i^i; r_m has positive degree.

    R = 0 gives (0, []); a constant R gives (R, [])."""
    r = zx_trim(int(c) for c in r)
    if not r:
        return 0, []
    u = content(r) * (1 if r[-1] > 0 else -1)
    a = tuple(c // u for c in r)
    if len(a) == 1:
        return u, []
    b = _deriv(a)
    g = gcd_z(a, b)
    c = zx_divexact(a, g)
    d = zx_sub(zx_divexact(b, g), _deriv(c))
    out = []
    while len(c) > 1:
        ri = gcd_z(c, d)
        c = zx_divexact(c, ri)
        d = zx_sub(zx_divexact(d, ri), _deriv(c))
        out.append(tuple(ri))
    return u, out
