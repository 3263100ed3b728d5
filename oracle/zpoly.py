"""Integer and integer-polynomial rings for the oracle (test infrastructure only).

Elements of Z[x] are tuples of Python ints, lowest power first, with no trailing
zeros; the zero polynomial is the empty tuple.  ``ZZ`` and ``ZX`` expose the same
five operations so that the determinant and remainder-sequence code in
``resultant.py`` is written once and runs over either ring.
"""

from __future__ import annotations

import math


def zx_trim(a) -> tuple:
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return tuple(a)


def zx_deg(a) -> int:
    return len(a) - 1          # -1 for the zero polynomial


def zx_add(a, b) -> tuple:
    n = max(len(a), len(b))
    return zx_trim([(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)])


def zx_neg(a) -> tuple:
    return tuple(-c for c in a)


def zx_sub(a, b) -> tuple:
    return zx_add(a, zx_neg(b))


def zx_mul(a, b) -> tuple:
    if not a or not b:
        return ()
    out = [0] * (len(a) + len(b) - 1)
    for i, c in enumerate(a):
        if c:
            for j, d in enumerate(b):
                out[i + j] += c * d
    return zx_trim(out)


def zx_eval(a, x: int) -> int:
    v = 0
    for c in reversed(a):
        v = v * x + c
    return v


def zx_divexact(a, b) -> tuple:
    """a / b in Z[x]; raises if b does not divide a exactly."""
    if not b:
        raise ZeroDivisionError("division by the zero polynomial")
    r = list(a)
    db = len(b) - 1
    lb = b[-1]
    if len(r) - 1 < db:
        if any(r):
            raise ArithmeticError("inexact polynomial division")
        return ()
    q = [0] * (len(r) - db)
    for k in range(len(r) - 1, db - 1, -1):
        c = r[k]
        if c == 0:
            continue
        if c % lb:
            raise ArithmeticError("inexact polynomial division")
        t = c // lb
        q[k - db] = t
        for i in range(db + 1):
            r[k - db + i] -= t * b[i]
    if any(r):
        raise ArithmeticError("inexact polynomial division")
    return zx_trim(q)


def content(a) -> int:
    g = 0
    for c in a:
        g = math.gcd(g, c)
    return g


def primitive_part(a) -> tuple:
    """a / content(a), sign chosen so the leading coefficient is positive."""
    a = zx_trim(a)
    if not a:
        return ()
    g = content(a)
    if a[-1] < 0:
        g = -g
    return tuple(c // g for c in a)


class _Ring:
    """The five operations the generic elimination code needs."""

    zero = None
    one = None

    def add(self, a, b): ...
    def sub(self, a, b): ...
    def mul(self, a, b): ...
    def divexact(self, a, b): ...
    def is_zero(self, a): ...


class _IntRing(_Ring):
    zero = 0
    one = 1

    def add(self, a, b):
        return a + b

    def sub(self, a, b):
        return a - b

    def mul(self, a, b):
        return a * b

    def divexact(self, a, b):
        q, r = divmod(a, b)
        if r:
            raise ArithmeticError("inexact integer division")
        return q

    def is_zero(self, a):
        return a == 0

    def neg(self, a):
        return -a


class _PolyRing(_Ring):
    zero = ()
    one = (1,)

    def add(self, a, b):
        return zx_add(a, b)

    def sub(self, a, b):
        return zx_sub(a, b)

    def mul(self, a, b):
        return zx_mul(a, b)

    def divexact(self, a, b):
        return zx_divexact(a, b)

    def is_zero(self, a):
        return len(a) == 0

    def neg(self, a):
        return zx_neg(a)


ZZ = _IntRing()
ZX = _PolyRing()
