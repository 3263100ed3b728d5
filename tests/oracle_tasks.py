"""Oracle work for the full-size GPU parity tests, run on every host core.

The functions here take one picklable work item each (inputs as lists or int64
arrays, evaluation points as Python ints) and call only ``oracle/``; the pool is
started with the ``spawn`` method, so it is safe whether or not the parent
process has already initialised CUDA.  Nothing here computes what the library
computes: it only hands the oracle its inputs and checks the defining
properties of a gcd over Z.
"""

from __future__ import annotations

import math
import multiprocessing as mp
import os

import oracle as O


def pool(processes: int | None = None):
    """A spawn-context pool with one worker per host core (or `processes`)."""
    return mp.get_context("spawn").Pool(processes or os.cpu_count() or 1)


def res_points(item):
    """(f, g, points) -> [R(a) for a in points], R = res_y(f, g), exact."""
    f, g, pts = item
    return [O.res_at_prs(f, g, a) for a in pts]


def res_full(item):
    """(f, g) -> every coefficient of res_y(f, g) (exact evaluation/interpolation)."""
    f, g = item
    return list(O.res_evalz(f, g))


def disc_full(f):
    """f -> every coefficient of res_y(f, f_y)."""
    return list(O.disc_res(f, "evalz"))


def gcd_exact(item):
    """(p, q) -> gcd(p, q) in Z[x] (primitive remainder sequence)."""
    p, q = item
    return list(O.gcd_z(p, q))


def coprime_mod(a, b, p: int = (1 << 61) - 1) -> bool:
    """True when a and b are coprime modulo the prime p and p divides neither leading
    coefficient; this proves them coprime over Q (a common factor over Z of positive
    degree has a leading coefficient dividing both, so it keeps its degree mod p and
    would divide both there)."""
    a = [x % p for x in a]
    b = [x % p for x in b]
    if not a or not b or a[-1] == 0 or b[-1] == 0:
        return False
    while b:
        while b and b[-1] == 0:
            b.pop()
        if not b:
            break
        inv = pow(b[-1], p - 2, p)
        while len(a) >= len(b):
            c = a[-1] * inv % p
            s = len(a) - len(b)
            for i in range(len(b)):
                a[s + i] = (a[s + i] - c * b[i]) % p
            a.pop()
            while a and a[-1] == 0:
                a.pop()
        a, b = b, a
    return len(a) == 1


def gcd_is_gcd(item) -> bool:
    """(p, q, g): g is gcd(p, q) over Z with the library's normalisation, checked by its
    defining properties instead of recomputing it: g divides p and q exactly, the
    cofactors are coprime over Q, cont(g) = gcd(cont p, cont q) and lc(g) > 0 (for
    p = q = 0: g = 0)."""
    p, q, g = item
    p, q = O.zx_trim(int(c) for c in p), O.zx_trim(int(c) for c in q)
    g = O.zx_trim(int(c) for c in g)
    if not p and not q:
        return not g
    if not g or g[-1] <= 0:
        return False
    if O.content(g) != math.gcd(O.content(p) if p else 0, O.content(q) if q else 0):
        return False
    if not (O.divides_z(g, p) and O.divides_z(g, q)):
        return False
    if not p or not q:
        return len(g) - 1 == len(p or q) - 1
    cp, cq = O.zx_divexact(p, g), O.zx_divexact(q, g)
    if len(cp) == 1 or len(cq) == 1:
        return True
    return coprime_mod(list(cp), list(cq))


def bound_interval(item):
    """(f, g or None) -> exact enclosure of log2 of the Hadamard bound of res_y(f, g)
    (g = None: res_y(f, f_y)); None for an empty Sylvester column."""
    from oracle.bound import resultant_bound_log2

    f, g = item
    if g is None:
        g = O.deriv_y(f)
    return resultant_bound_log2(f, g)
