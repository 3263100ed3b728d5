"""Seeded synthetic inputs for the resultant and gcd workloads.

This module only draws random integers and assembles polynomials from them.  It
contains none of the resultant or gcd arithmetic: the CPU oracle and the CUDA
path both receive their inputs from here, and nothing else is shared between
them.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state_i = key + i * 0x9E3779B97F4A7C15,
followed by the published two-multiply finaliser.  It is written out here so the
streams are identical on every machine and numpy version.

Polynomial conventions used everywhere in this package:

* a bivariate polynomial f in Z[x, y] is a list of rows ``f[j][i]`` = coefficient
  of x^i y^j (rows indexed by the power of y, columns by the power of x); the
  helper :func:`to_array` turns it into a dense int64 numpy array when every
  coefficient fits, else an object array of Python ints;
* a univariate polynomial is a list ``p[i]`` = coefficient of x^i.

The shapes follow the paper's test families (Section 4, "Implementation and
Experiments": dense random curves, products of circles/ellipses such as
"ten_circles") because the paper's own data sets are not available.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream keyed by (seed, stream id)."""

    def __init__(self, seed: int, stream: int = 0):
        with np.errstate(over="ignore"):
            k = _splitmix(np.array([(seed * 0x100000001B3 + stream) & (2**64 - 1)], dtype=np.uint64))
        self.key = k[0]
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.ctr + 1, self.ctr + n + 1, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _splitmix(self.key + idx * _GOLDEN)

    def signed_bits(self, bits: int, n: int) -> list[int]:
        """n integers uniform in [-2^(bits-1), 2^(bits-1) - 1] (exactly uniform: top bits)."""
        assert 1 <= bits <= 64
        u = self.u64(n) >> np.uint64(64 - bits)
        half = 1 << (bits - 1)
        return [int(v) - half for v in u.tolist()]

    def uniform_int(self, lo: int, hi: int, n: int) -> list[int]:
        """n integers uniform in [lo, hi] (multiply-shift on 32 bits; span <= 2^32)."""
        span = hi - lo + 1
        assert 1 <= span <= 2**32
        u = (self.u64(n) >> np.uint64(32)).astype(object)
        return [lo + (int(v) * span >> 32) for v in u]

    def uniform01(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)


# --------------------------------------------------------------------------- helpers


def to_array(rows: list[list[int]], dx: int | None = None, dy: int | None = None) -> np.ndarray:
    """Dense [y][x] array of a bivariate polynomial; int64 when every entry fits."""
    dy = len(rows) - 1 if dy is None else dy
    dx = max(len(r) for r in rows) - 1 if dx is None else dx
    big = any(c < -(2**63) or c >= 2**63 for r in rows for c in r)
    out = np.zeros((dy + 1, dx + 1), dtype=object if big else np.int64)
    if big:
        out[:, :] = 0
    for j, r in enumerate(rows):
        for i, c in enumerate(r):
            out[j, i] = c
    return out


def _mul2(a: list[list[int]], b: list[list[int]]) -> list[list[int]]:
    """Product of two bivariate polynomials (input construction only)."""
    ay, by = len(a), len(b)
    ax = max(len(r) for r in a)
    bx = max(len(r) for r in b)
    out = [[0] * (ax + bx - 1) for _ in range(ay + by - 1)]
    for j1, r1 in enumerate(a):
        for i1, c1 in enumerate(r1):
            if c1:
                for j2, r2 in enumerate(b):
                    orow = out[j1 + j2]
                    for i2, c2 in enumerate(r2):
                        if c2:
                            orow[i1 + i2] += c1 * c2
    return out


def _mul1(a: list[int], b: list[int]) -> list[int]:
    out = [0] * (len(a) + len(b) - 1)
    for i, c in enumerate(a):
        if c:
            for j, d in enumerate(b):
                out[i + j] += c * d
    return out


def dense_total_degree(st: Stream, d: int, bits: int) -> list[list[int]]:
    """Dense f with every monomial x^i y^j, i + j <= d, coefficients signed `bits`-bit."""
    n = (d + 1) * (d + 2) // 2
    c = st.signed_bits(bits, n)
    rows, t = [], 0
    for j in range(d + 1):
        rows.append(c[t:t + d + 1 - j] + [0] * j)
        t += d + 1 - j
    return rows


def dense_box(st: Stream, dx: int, dy: int, bits: int) -> list[list[int]]:
    """Dense f with every monomial x^i y^j, i <= dx, j <= dy."""
    c = st.signed_bits(bits, (dx + 1) * (dy + 1))
    return [c[j * (dx + 1):(j + 1) * (dx + 1)] for j in range(dy + 1)]


def _nonzero(st: Stream, bits: int) -> int:
    while True:
        v = st.signed_bits(bits, 1)[0]
        if v:
            return v


# --------------------------------------------------------------------------- configs


@dataclass
class PairSet:
    """A list of bivariate pairs (f, g) plus metadata for the batch."""

    f: list = field(default_factory=list)
    g: list = field(default_factory=list)
    planted: list = field(default_factory=list)
    info: dict = field(default_factory=dict)


def small_dense_pair(seed: int = 1, d: int = 6, bits: int = 8):
    """One dense pair of total degree d with coefficients in [-2^(bits-1), 2^(bits-1)-1]
    (degree 6, [-128, 127] is the single-pair workload)."""
    st = Stream(seed, 0)
    f = dense_total_degree(st, d, bits)
    g = dense_total_degree(st, d, bits)
    return f, g


def deg20_pair(seed: int = 2, d: int = 20, bits: int = 16):
    """Dense total-degree-20 f and an independent g, 16-bit signed coefficients."""
    return small_dense_pair(seed, d, bits)


def deg20_batch(n: int = 4096, base_seed: int = 2000, d: int = 20, bits: int = 16) -> PairSet:
    """The batched degree-20 workload: pair i uses seed base_seed + i."""
    ps = PairSet(info=dict(d=d, bits=bits, base_seed=base_seed))
    for i in range(n):
        f, g = small_dense_pair(base_seed + i, d, bits)
        ps.f.append(f)
        ps.g.append(g)
        ps.planted.append(False)
    return ps


def deg20_batch_arrays(n: int = 4096, base_seed: int = 2000, d: int = 20, bits: int = 16):
    """Same inputs as :func:`deg20_batch` as int64 arrays [n][d+1][d+1] (fast path)."""
    m = (d + 1) * (d + 2) // 2
    jj, ii = [], []
    for j in range(d + 1):
        for i in range(d + 1 - j):
            jj.append(j)
            ii.append(i)
    F = np.zeros((n, d + 1, d + 1), dtype=np.int64)
    G = np.zeros((n, d + 1, d + 1), dtype=np.int64)
    half = np.int64(1 << (bits - 1))
    for k in range(n):
        st = Stream(base_seed + k, 0)
        u = (st.u64(2 * m) >> np.uint64(64 - bits)).astype(np.int64) - half
        F[k, jj, ii] = u[:m]
        G[k, jj, ii] = u[m:]
    return F, G


def mixed_batch(seed: int = 3, n: int = 4096, planted_frac: float = 0.25) -> PairSet:
    """Heterogeneous batch: per pair deg_x, deg_y ~ U{4..16} (shared by f and g),
    coefficient bits ~ U{8..32}; a quarter of the pairs share a planted factor h of
    total degree U{1..3} with deg_y h >= 1 and 8-bit coefficients (their resultant is 0)."""
    st = Stream(seed, 0)
    ps = PairSet(info=dict(kind="mixed"))
    for _ in range(n):
        dx, dy = st.uniform_int(4, 16, 2)
        bits = st.uniform_int(8, 32, 1)[0]
        plant = st.uniform01(1)[0] < planted_frac
        if plant:
            t = st.uniform_int(1, 3, 1)[0]
            h = dense_total_degree(st, t, 8)
            if h[t][0] == 0:
                h[t][0] = _nonzero(st, 8)
            f = _mul2(h, dense_box(st, dx - t, dy - t, bits))
            g = _mul2(h, dense_box(st, dx - t, dy - t, bits))
        else:
            f = dense_box(st, dx, dy, bits)
            g = dense_box(st, dx, dy, bits)
        ps.f.append(f)
        ps.g.append(g)
        ps.planted.append(plant)
    return ps


def gcd_batch(seed: int = 3, n: int = 4096, lo: int = 30, hi: int = 200, hdeg: int = 5):
    """Univariate gcd jobs P = h*u, Q = h*v with deg P, deg Q ~ U{lo..hi}, deg h = hdeg;
    h has 8-bit coefficients, u and v have U{8..32}-bit coefficients."""
    st = Stream(seed, 1)
    P, Q, H = [], [], []
    for _ in range(n):
        dp, dq = st.uniform_int(lo, hi, 2)
        bits = st.uniform_int(8, 32, 1)[0]
        h = st.signed_bits(8, hdeg + 1)
        if h[-1] == 0:
            h[-1] = _nonzero(st, 8)
        u = st.signed_bits(bits, dp - hdeg + 1)
        v = st.signed_bits(bits, dq - hdeg + 1)
        if u[-1] == 0:
            u[-1] = _nonzero(st, bits)
        if v[-1] == 0:
            v[-1] = _nonzero(st, bits)
        P.append(_mul1(h, u))
        Q.append(_mul1(h, v))
        H.append(h)
    return P, Q, H


def sqf_batch(seed: int = 6, n: int = 2048, degs=((20, 60), (4, 16), (0, 4)), bits: int = 16,
              unit_bits: int = 8):
    """Square-free factorisation inputs R = u * r_1 * r_2^2 * r_3^3 ... shaped like the
    projection resultants res(f, f_y) of curves with nodes and cusps: a large
    square-free part, squared factors from the singular points, a few higher powers.
    deg r_i ~ U{degs[i-1]}, coefficients signed `bits`-bit (non-zero leading term),
    u a signed `unit_bits`-bit constant.  Returns (R list, planted list of (u, [r_i]))."""
    st = Stream(seed, 2)
    R, planted = [], []
    for _ in range(n):
        u = _nonzero(st, unit_bits)
        facs = []
        for lo, hi in degs:
            d = st.uniform_int(lo, hi, 1)[0]
            r = st.signed_bits(bits, d + 1)
            if r[-1] == 0:
                r[-1] = _nonzero(st, bits)
            facs.append(r)
        out = [u]
        for i, r in enumerate(facs, start=1):
            for _ in range(i):
                out = _mul1(out, r)
        R.append(out)
        planted.append((u, facs))
    return R, planted


def conic_curves(seed: int = 4, ncon: int = 8, rbits: int = 10, nterms: int = 16,
                 tdeg: int = 16, tbits: int = 32, gdeg: int = 24, gbits: int = 64):
    """Large structured curves: f = product of `ncon` circles/axis-parallel ellipses with
    integer centres and radii in [-2^rbits, 2^rbits] (radii non-zero), plus `nterms`
    random monomials x^i y^j, i + j <= tdeg, with `tbits`-bit coefficients; g dense of
    total degree `gdeg` with `gbits`-bit coefficients."""
    st = Stream(seed, 0)
    lim = 1 << rbits
    f = [[1]]
    for _ in range(ncon):
        kind = st.uniform_int(0, 1, 1)[0]
        a, b = st.uniform_int(-lim, lim, 2)
        if kind == 0:
            r = 0
            while r == 0:
                r = st.uniform_int(-lim, lim, 1)[0]
            # (x-a)^2 + (y-b)^2 - r^2
            c = [[a * a + b * b - r * r, -2 * a, 1], [-2 * b, 0, 0], [1, 0, 0]]
        else:
            A = B = 0
            while A == 0:
                A = st.uniform_int(-lim, lim, 1)[0]
            while B == 0:
                B = st.uniform_int(-lim, lim, 1)[0]
            A2, B2 = A * A, B * B
            # B^2 (x-a)^2 + A^2 (y-b)^2 - A^2 B^2
            c = [[B2 * a * a + A2 * b * b - A2 * B2, -2 * B2 * a, B2], [-2 * A2 * b, 0, 0], [A2, 0, 0]]
        f = _mul2(f, c)
    for _ in range(nterms):
        j = st.uniform_int(0, tdeg, 1)[0]
        i = st.uniform_int(0, tdeg - j, 1)[0]
        f[j][i] += st.signed_bits(tbits, 1)[0]
    g = dense_total_degree(st, gdeg, gbits)
    return f, g


def arrangement_curves(seed: int = 7, n: int = 90, d: int = 8, bits: int = 12, conic_frac: float = 0.25,
                       rbits: int = 6):
    """An arrangement of n curves for the curve-pair analysis (Section 3): a fraction
    `conic_frac` are products of d/2 circles/axis-parallel ellipses with integer centres
    and radii in [-2^rbits, 2^rbits] (singular where the conics meet, like the paper's
    circle families), the others dense random curves of total degree d with `bits`-bit
    coefficients (non-zero y^d term, so the y-degree is d)."""
    st = Stream(seed, 3)
    curves = []
    for _ in range(n):
        if st.uniform01(1)[0] < conic_frac:
            f, _g = conic_curves(int(st.u64(1)[0] >> np.uint64(33)), ncon=max(1, d // 2), rbits=rbits, nterms=0,
                                 gdeg=1, gbits=2)
        else:
            f = dense_total_degree(st, d, bits)
            if f[d][0] == 0:
                f[d][0] = _nonzero(st, bits)
        curves.append(f)
    return curves


@dataclass
class Request:
    t_arrive: float
    kind: str            # "res" or "gcd"
    a: list
    b: list
    planted: bool


def serving_stream(seed: int = 5, n: int = 100_000, rate: float = 1000.0, planted_frac: float = 0.10,
                   dlo: int = 5, dhi: int = 30, blo: int = 8, bhi: int = 64):
    """Poisson-arrival stream of mixed resultant / gcd requests.  Degree is
    round(exp(U(ln dlo, ln dhi))), coefficient bits U{blo..bhi}; a tenth carry a planted
    common factor (resultant: bivariate h with deg_y h >= 1; gcd: degree 1..3).  Every
    coefficient of a request fits in a signed 64-bit word: the cofactor of a planted
    factor draws fewer bits so the product stays inside the request's bit budget."""
    st = Stream(seed, 0)
    out = []
    t = 0.0
    for _ in range(n):
        u = st.uniform01(3)
        t += -math.log(1.0 - u[0]) / rate
        kind = "res" if u[1] < 0.5 else "gcd"
        d = int(round(math.exp(math.log(dlo) + (math.log(dhi) - math.log(dlo)) * st.uniform01(1)[0])))
        bits = st.uniform_int(blo, bhi, 1)[0]
        plant = u[2] < planted_frac
        if kind == "res":
            if plant:
                hd = st.uniform_int(1, min(3, d - 1), 1)[0]
                h = dense_total_degree(st, hd, 4)
                if h[hd][0] == 0:
                    h[hd][0] = _nonzero(st, 4)
                cb = max(2, bits - 4 - 2 * (hd + 2).bit_length() - 2)
                a = _mul2(h, dense_total_degree(st, d - hd, cb))
                b = _mul2(h, dense_total_degree(st, d - hd, cb))
            else:
                a = dense_total_degree(st, d, bits)
                b = dense_total_degree(st, d, bits)
        else:
            if plant:
                hd = st.uniform_int(1, min(3, d - 1), 1)[0]
                h = st.signed_bits(4, hd + 1)
                if h[-1] == 0:
                    h[-1] = _nonzero(st, 4)
                cb = max(2, bits - 4 - (hd + 1).bit_length() - 2)
                a = _mul1(h, st.signed_bits(cb, d - hd + 1))
                b = _mul1(h, st.signed_bits(cb, d - hd + 1))
            else:
                a = st.signed_bits(bits, d + 1)
                b = st.signed_bits(bits, d + 1)
        out.append(Request(t, kind, a, b, plant))
    return out


def planted_roots_pair(seed: int, m: int, n: int, bits: int = 6, lc_bits: int = 4):
    """f = a * prod_i (y - alpha_i(x)), g = b * prod_j (y - beta_j(x)) with alpha, beta
    linear in x; returns (f, g, alphas, betas, a, b) where each alpha is [c0, c1]."""
    st = Stream(seed, 7)
    al = [st.signed_bits(bits, 2) for _ in range(m)]
    be = [st.signed_bits(bits, 2) for _ in range(n)]
    a = _nonzero(st, lc_bits)
    b = _nonzero(st, lc_bits)
    f = [[a]]
    for r in al:
        f = _mul2(f, [[-r[0], -r[1]], [1]])
    g = [[b]]
    for r in be:
        g = _mul2(g, [[-r[0], -r[1]], [1]])
    return f, g, al, be, a, b
