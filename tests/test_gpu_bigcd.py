"""GPU parity: gcd cofactors, the gcd in Z[x][y] with cofactors and the Teissier
resultant Q = res(f_x/h, f_y/h, y), h = gcd(f_x, f_y) (Section 2.1), against the
CPU oracle (gcd_z / zx_divexact, gcd_zxy / divexact_zxy, teissier_q).  Exact.
"""

import random

import pytest

import oracle as O
from paper_1103_4697_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1103_4697_gb300.api import Context

    c = Context(device=0, mem_budget=4 << 30)
    yield c
    c.close()


def _trim(a):
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def _rows(rows):
    """Oracle rows (tuples, trimmed) as the binding returns them: lists, each row padded
    to the polynomial's x-degree."""
    rows = [list(r) for r in rows]
    if not rows:
        return []
    w = max(len(r) for r in rows)
    return [r + [0] * (w - len(r)) for r in rows]


def _mul2(a, b):
    out = [[0] * (max(len(r) for r in a) + max(len(r) for r in b) - 1) for _ in range(len(a) + len(b) - 1)]
    for j1, r1 in enumerate(a):
        for i1, c1 in enumerate(r1):
            if c1:
                for j2, r2 in enumerate(b):
                    for i2, c2 in enumerate(r2):
                        out[j1 + j2][i1 + i2] += c1 * c2
    return out


def _rand2(rng, dy, dx, amp):
    f = [[rng.randint(-amp, amp) for _ in range(dx + 1)] for _ in range(dy + 1)]
    f[dy][rng.randint(0, dx)] = rng.choice([1, -1, 2, 3])
    return f


def test_gcd_cofactors(ctx):
    P, Q, _ = W.gcd_batch(31, 40, lo=5, hi=40, hdeg=4)
    P += [[0], [0], [3, 0, -6], [5], [0, 0, 4]]
    Q += [[0], [2, -4, 6], [0], [10, 0, 5], [0, 2]]
    got = ctx.gcd_cofactors_batch(P, Q)
    for p, q, (g, a, b) in zip(P, Q, got):
        want = list(O.gcd_z(p, q))
        assert g == want
        if not want:
            assert a == [] and b == []
            continue
        assert a == list(O.zx_divexact(O.zx_trim(p), tuple(want)))
        assert b == list(O.zx_divexact(O.zx_trim(q), tuple(want)))


def test_gcd2_hand_cases(ctx):
    xpy, xmy = [[0, 1], [1]], [[0, 1], [-1]]
    cases = [
        ([[0, 0], [0, 1]], [[0, 0, 1]]),                 # gcd(x y, x^2) = x
        (_mul2(xpy, xpy), _mul2(xpy, xmy)),              # x + y
        (xpy, xmy),                                      # images share z, the gcd is 1
        (_mul2(_mul2(xpy, [[0, 1]]), [[0], [1]]), _mul2(xmy, [[0, 1], [0, 1]])),   # monomial factors
        ([[0]], [[0, 0], [0, 3]]),                       # gcd(0, 3 x y)
        ([[6, 4], [2]], [[9, 6], [3]]),                  # contents 2 and 3, common part
        # both vanish at (1, 1) outside their gcd: every monomial substitution keeps
        # z - 1 in the images, so the library shifts y -> y + s
        ([[0, -3], [-3, 0], [0, 4], [4, -1], [-1, 0]],
         [[0, 9, 12, -9], [-9, -6, 9, -12], [-6, 6, 2, 0], [-6, 23, 10, 1], [-13, -14, -3, 0], [4, 2, 0, 0]]),
    ]
    got = ctx.gcd2_batch([c[0] for c in cases], [c[1] for c in cases])
    for (f, g), (h, a, b) in zip(cases, got):
        H = O.gcd_zxy(f, g)
        assert h == _rows(H), (f, g)
        if H:
            assert a == _rows(O.divexact_zxy(f, H))
            assert b == _rows(O.divexact_zxy(g, H))


@pytest.mark.parametrize("seed", range(6))
def test_gcd2_planted(ctx, seed):
    rng = random.Random(5100 + seed)
    fs, gs = [], []
    for _ in range(12):
        h = _rand2(rng, rng.randint(0, 2), rng.randint(0, 2), 4)
        u = _rand2(rng, rng.randint(0, 3), rng.randint(0, 3), 9)
        v = _rand2(rng, rng.randint(0, 3), rng.randint(0, 3), 9)
        fs.append(_mul2(h, u))
        gs.append(_mul2(h, v))
    got = ctx.gcd2_batch(fs, gs)
    for f, g, (h, a, b) in zip(fs, gs, got):
        H = O.gcd_zxy(f, g)
        assert h == _rows(H)
        assert a == _rows(O.divexact_zxy(f, H)) and b == _rows(O.divexact_zxy(g, H))


def test_teissier_q(ctx):
    rng = random.Random(52)
    xpy = [[0, 1], [1]]
    curves = []
    f = _mul2(xpy, xpy)
    f[0][0] += 1
    curves.append(f)                                     # (x + y)^2 + 1: h = 2x + 2y, Q = 1
    curves.append([[0, 0, -1, -1], [0], [1]])            # y^2 - x^2 - x^3: a node at the origin
    L = [[0, 1], [2]]
    g = [[rng.randint(-3, 3)]]
    p = [[1]]
    for k in range(1, 4):                                # a polynomial in x + 2y
        p = _mul2(p, L)
        c = rng.randint(-3, 3) or 1
        g = [[(g[j][i] if j < len(g) and i < len(g[j]) else 0) + c * (p[j][i] if j < len(p) and i < len(p[j]) else 0)
              for i in range(max(len(r) for r in g + p))] for j in range(max(len(g), len(p)))]
    curves.append(g)
    c1, _ = W.conic_curves(9, ncon=2, rbits=3, nterms=0)
    curves.append(c1)                                    # two circles / ellipses
    for _ in range(3):
        curves.append(_rand2(rng, 3, 3, 6))              # generic: h is a constant
    got = ctx.teissier_res_batch(curves)
    for f, q in zip(curves, got):
        assert q == list(O.teissier_q(f)), f


def _transpose(f):
    w = max(len(r) for r in f)
    rows = [list(r) + [0] * (w - len(r)) for r in f]
    return [[rows[j][i] for j in range(len(rows))] for i in range(w)]


def test_content(ctx):
    """Content removal (Section 2): gcd of the coefficients of the powers of y (and of
    x, on the transposed curve), against the oracle's content_y."""
    rng = random.Random(53)
    curves = []
    for _ in range(20):
        h = [[rng.randint(-4, 4) for _ in range(rng.randint(1, 3))]]   # a factor in x alone
        if not any(h[0]):
            h[0][0] = 3
        curves.append(_mul2(h, _rand2(rng, rng.randint(0, 3), rng.randint(0, 3), 9)))
    curves += [[[0, 0], [0, 0]], [[5, 0, 10]], [[0, 3], [0, 6], [0, 9]], [[-4, 0, 2]], _rand2(rng, 2, 2, 5)]
    got = ctx.content_batch(curves)
    for f, g in zip(curves, got):
        assert g == list(O.content_y(f)), f
    got0 = ctx.content_batch(curves, var=0)
    for f, g in zip(curves, got0):
        assert g == list(O.content_y(_transpose(f))), f
