"""GPU parity at the documented size limits of the C ABI (include/gbres.h).

Covered: the largest y-degree (GBR_MAX_YDEG = 127), the widest input coefficients
(GBR_MAX_WORDS = 8 words), an x-degree bound near GBR_MAX_POINTS (default and
drop modes), results wider than 1280 limbs (between 1321 and GBR_MAX_PRIMES =
2048 primes), and gcd inputs of degree GBR_MAX_UDEG = 8191.  One step beyond a
limit the call is refused with GBR_ELIMIT or GBR_EINVAL.  Large results are
checked by their exact values R(a) against the oracle's at sampled integer
points where both leading coefficients are non-zero.  Small ones are checked
coefficient by coefficient, and the gcd by a closed form:
gcd(h (x^a - 1), h (x^b - 1)) = h (x - 1) for coprime a, b and primitive h.
"""

import random

import pytest

import oracle as O
from oracle.resultant import as_zxy
from paper_1103_4697_gb300 import native as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1103_4697_gb300.api import Context

    c = Context(device=0, mem_budget=4 << 30)
    yield c
    c.close()


def _rows(rng, dy, dx, amp):
    rows = [[rng.randint(-amp, amp) for _ in range(dx + 1)] for _ in range(dy + 1)]
    rows[dy][dx] = amp                                   # full degree in both variables
    return rows


def _ev(r, a):
    v = 0
    for c in reversed(r):
        v = v * a + c
    return v


def _points(f, g, cands):
    """The candidate points where lc_y f and lc_y g do not vanish (the oracle's
    integer subresultant sequence applies there)."""
    lf, lg = as_zxy(f)[-1], as_zxy(g)[-1]
    return [a for a in cands if O.zx_eval(lf, a) != 0 and O.zx_eval(lg, a) != 0]


def _mul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return out


def test_largest_y_degree(ctx):
    rng = random.Random(81)
    f, g = _rows(rng, 127, 1, 3), _rows(rng, 127, 1, 3)
    r = ctx.resultant(f, g)
    assert len(r) - 1 <= 254
    pts = _points(f, g, [2, -2, 5, rng.randint(-10 ** 6, 10 ** 6)])
    assert len(pts) >= 3
    for a in pts:
        assert _ev(r, a) == O.res_at_prs(f, g, a)
    d = ctx.discriminant_res(f)
    fy = O.deriv_y(f)
    for a in _points(f, fy, [3, rng.randint(-10 ** 6, 10 ** 6)]):
        assert _ev(d, a) == O.res_at_prs(f, fy, a)
    with pytest.raises(N.GbrError) as e:
        ctx.resultant(_rows(rng, 128, 1, 3), g)
    assert e.value.status == N.ELIMIT


def test_widest_input_coefficients(ctx):
    rng = random.Random(82)
    big = (1 << 511) - 1                                  # 8 two's-complement words
    f, g = _rows(rng, 3, 2, big), _rows(rng, 2, 3, big)
    assert ctx.resultant(f, g) == list(O.res_subres(f, g))
    assert ctx.resultant(g, f, var=0) == list(O.res_subres(_transpose(g), _transpose(f)))
    f9 = [list(r) for r in f]
    f9[1][1] = 1 << 511                                   # 9 words
    with pytest.raises(N.GbrError) as e:
        ctx.resultant(f9, g)
    assert e.value.status == N.EINVAL


def _transpose(f):
    w = max(len(r) for r in f)
    rows = [list(r) + [0] * (w - len(r)) for r in f]
    return [[rows[j][i] for j in range(len(rows))] for i in range(w)]


def test_results_wider_than_1280_limbs(ctx):
    """Between 1321 and 2048 primes: the Chinese remaindering of such results runs
    with blocks narrower than a warp (about 59 000-bit coefficients)."""
    from paper_1103_4697_gb300.api import resultant_info

    rng = random.Random(83)
    big = (1 << 511) - 1
    f, g = _rows(rng, 56, 1, big), _rows(rng, 56, 1, big)
    info = resultant_info(f, g)
    assert 1321 < info["primes"] <= 2048
    r = ctx.resultant(f, g)
    assert len(r) - 1 <= info["deg_bound"]
    assert max(abs(c).bit_length() for c in r) <= info["log2_bound"] + 1
    for a in _points(f, g, [2, -3])[:2]:
        assert _ev(r, a) == O.res_at_prs(f, g, a)
    with pytest.raises(N.GbrError) as e:                  # more than GBR_MAX_PRIMES
        ctx.resultant(_rows(rng, 64, 1, big), _rows(rng, 64, 1, big))
    assert e.value.status == N.ELIMIT


def test_x_degree_bound_near_the_point_limit(ctx):
    """D = 16000 (16001 of the 16384 points) with leading coefficients of degree
    4000: the default choice (roots of unity, N = 16384, inverse transform), the
    symmetric integer points (Newton interpolation) and the drop mode (Newton on
    the integer grid with 8000 spare points) give the same result."""
    from paper_1103_4697_gb300.native import OPT_DROP_UNLUCKY, OPT_POINTS, OPT_STATS

    rng = random.Random(84)
    f, g = _rows(rng, 2, 4000, 3), _rows(rng, 2, 4000, 3)
    ctx.set_option(OPT_STATS, 1)
    r0 = ctx.resultant(f, g)
    assert ctx.stats()["root_pairs"] == 1
    ctx.set_option(OPT_POINTS, 1)
    try:
        r2 = ctx.resultant(f, g)
        assert ctx.stats()["root_pairs"] == 0
    finally:
        ctx.set_option(OPT_POINTS, 0)
    ctx.set_option(OPT_DROP_UNLUCKY, 1)
    try:
        r1 = ctx.resultant(f, g)
    finally:
        ctx.set_option(OPT_DROP_UNLUCKY, 0)
    assert r0 == r1 == r2
    assert len(r0) - 1 <= 16000
    for a in _points(f, g, [0, 1, -1, 7, rng.randint(-10 ** 6, 10 ** 6)]):
        assert _ev(r0, a) == O.res_at_prs(f, g, a)
    with pytest.raises(N.GbrError) as e:                  # D = 16800: above GBR_MAX_POINTS - 1
        ctx.resultant(_rows(rng, 2, 4200, 3), _rows(rng, 2, 4200, 3))
    assert e.value.status == N.ELIMIT


def test_gcd_at_the_largest_degree(ctx):
    """P = h (x^8186 - 1) of degree 8191, Q = h (x^8185 - 1): gcd h (x - 1) and
    cofactors 1 + x + ... + x^8185 and 1 + x + ... + x^8184."""
    rng = random.Random(85)
    h = [1] + [rng.randint(-128, 127) for _ in range(4)] + [rng.randint(1, 127)]   # primitive, lc > 0
    P = _mul(h, [-1] + [0] * 8185 + [1])
    Q = _mul(h, [-1] + [0] * 8184 + [1])
    assert len(P) - 1 == 8191
    (g, a, b), = ctx.gcd_cofactors_batch([P], [Q])
    assert g == _mul(h, [-1, 1])
    assert a == [1] * 8186 and b == [1] * 8185
    with pytest.raises(N.GbrError) as e:
        ctx.gcd(_mul(h, [-1] + [0] * 8186 + [1]), Q)      # degree 8192
    assert e.value.status == N.ELIMIT
