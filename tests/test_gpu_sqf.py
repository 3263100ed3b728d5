"""GPU parity: the square-free factorisation R = u * prod r_i^i (Section 2.1,
Projection Phase) from libgbres equals the CPU oracle's Yun factorisation
exactly (integer results, tolerance 0).

Small and ragged cases compare (u, [r_1..r_m]) element by element with
oracle.sqf_yun.  The full-size batch compares sampled jobs with the oracle and
checks every job by properties that fix the answer: the product u prod r_i^i
equals R, every r_i is primitive with a positive leading coefficient, and the
degree pattern is the planted one (the planted factors are square-free and
pairwise coprime for this seed, which the sampled oracle comparisons confirm).
"""

import math
import random

import pytest

import oracle as O
from paper_1103_4697_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1103_4697_gb300.api import Context

    c = Context(device=0, mem_budget=8 << 30)
    yield c
    c.close()


def _oracle(r):
    u, fs = O.sqf_yun(r)
    return u, [list(f) for f in fs]


def _mul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return out


def _trim(a):
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def _expand(u, fs):
    out = [u]
    for i, f in enumerate(fs, start=1):
        for _ in range(i):
            out = _mul(out, f)
    return _trim(out)


def test_hand_cases(ctx):
    cases = [
        [-3, 6, -3],          # -3 (x - 1)^2
        [0, 0, 0, 4],         # 4 x^3: r_1 = r_2 = 1, r_3 = x
        [-2, 0, 2],           # 2 (x^2 - 1)
        [1, 1],               # x + 1
        [0, 5],               # 5 x
        [7, 0, 0, 0, 0, 0, 0],   # leading zeros: the constant 7
    ]
    for r in cases:
        assert ctx.squarefree(r) == _oracle(r), r


def test_zero_and_constants(ctx):
    assert ctx.squarefree([]) == (0, [])
    assert ctx.squarefree([0, 0]) == (0, [])
    assert ctx.squarefree([-6]) == (-6, [])
    assert ctx.squarefree([2**100 + 3]) == (2**100 + 3, [])


@pytest.mark.parametrize("seed", range(8))
def test_random_products(ctx, seed):
    rng = random.Random(1300 + seed)
    R = [rng.choice([1, -1, 2, -6, 35])]
    for _ in range(rng.randint(1, 5)):
        p = _trim([rng.randint(-20, 20) for _ in range(rng.randint(2, 6))]) or [1]
        for _ in range(rng.randint(1, 4)):
            R = _mul(R, p)
    assert ctx.squarefree(R) == _oracle(R)


def test_generic_square_free(ctx):
    # random dense R is square-free: one factor, the primitive part
    rng = random.Random(77)
    for d in (1, 2, 31, 32, 33, 100):
        r = [rng.randint(-2**40, 2**40) for _ in range(d + 1)]
        r[-1] = r[-1] or 1
        assert ctx.squarefree(r) == _oracle(r), d


def test_wide_coefficients(ctx):
    # content, several limbs, high multiplicity
    a = [3 * 2**70 + 1, -(2**65), 5]
    b = [-(2**90) - 7, 1]
    R = _mul(_mul(_mul(a, a), _mul(b, b)), b)
    R = [12345678901234567 * c for c in R]
    assert ctx.squarefree(R) == _oracle(R)
    R2 = _mul(R, [0, 0, 1])     # times x^2
    assert ctx.squarefree(R2) == _oracle(R2)


def test_square_free_test_path(ctx):
    # lifts of 12 or more primes first get the two-prime square-free test: wide
    # square-free inputs (with and without a content) finish there, wide inputs with
    # repeated factors fall through to the full lift
    rng = random.Random(31)
    cases = []
    for d in (1, 7, 40):
        r = [rng.randint(-2**400, 2**400) for _ in range(d + 1)]
        r[-1] = r[-1] or 1
        cases.append(r)
        cases.append([-(3**50) * c for c in r])                     # content 3^50, negative lc
    a = [rng.randint(-2**150, 2**150) for _ in range(6)]
    b = [rng.randint(-2**120, 2**120) for _ in range(4)]
    cases.append(_mul(_mul(a, a), b))                                 # a^2 b, about 420-bit coefficients
    cases.append(_mul(_mul(_mul(b, b), b), [0, 1]))                   # x b^3
    got = ctx.squarefree_batch(cases)
    assert got == [_oracle(r) for r in cases]


def test_high_multiplicity(ctx):
    for k in (5, 9, 17):
        R = [1]
        for _ in range(k):
            R = _mul(R, [-2, 3])
        R = _mul(R, [1, 0, 1])
        assert ctx.squarefree(R) == _oracle(R), k


def test_projection_resultant_two_circles(ctx):
    # R = res_y(F, F_y) of the union of two intersecting circles: the
    # intersection points give squared factors (computed by the oracle)
    def circle(a, b, r2):
        return [[a * a + b * b - r2, -2 * a, 1], [-2 * b, 0, 0], [1, 0, 0]]

    F = W._mul2(circle(0, 0, 25), circle(3, 1, 16))
    Fy = [[(j + 1) * c for c in F[j + 1]] for j in range(len(F) - 1)]
    R = _trim(O.res_subres(F, Fy))
    got = ctx.squarefree(R)
    assert got == _oracle(R)
    assert len(got[1]) >= 2 and len(got[1][1]) > 1     # a squared factor is present


def test_projection_resultant_three_conics(ctx):
    # a product of three circles/ellipses from the curve generator: R has a
    # squared factor for the intersection points and the x-extreme points
    f, _ = W.conic_curves(8, ncon=3, rbits=4, nterms=0)
    fy = [[(j + 1) * c for c in f[j + 1]] for j in range(len(f) - 1)]
    R = _trim(O.res_subres(f, fy))
    assert ctx.squarefree(R) == _oracle(R)


def test_batch_mixed(ctx):
    R, _ = W.sqf_batch(11, 24, degs=((0, 12), (0, 6), (0, 3)), bits=12)
    R = R + [[], [5], [0, 0, 3], [-1, 0, 1]]
    rng = random.Random(5)
    rng.shuffle(R)
    got = ctx.squarefree_batch(R)
    assert got == [_oracle(r) for r in R]


def test_batch_of_workload_shape(ctx):
    R, _ = W.sqf_batch(6, 16)
    got = ctx.squarefree_batch(R)
    assert got == [_oracle(r) for r in R]


def test_full_batch_properties_and_samples(ctx):
    R, planted = W.sqf_batch(6, 2048)
    got = ctx.squarefree_batch(R)
    assert len(got) == len(R)
    for r, (u, fs), (pu, pf) in zip(R, got, planted):
        assert _expand(u, fs) == _trim(r)
        for f in fs:
            assert f[-1] > 0 and math.gcd(*f) == 1
        want = [len(f) - 1 for f in pf]
        while want and want[-1] == 0:
            want.pop()
        assert [len(f) - 1 for f in fs] == want
    for k in random.Random(9).sample(range(len(R)), 6):
        assert got[k] == _oracle(R[k]), k


def test_batch_determinism(ctx):
    R, _ = W.sqf_batch(12, 64, degs=((5, 20), (1, 6), (0, 2)), bits=24)
    assert ctx.squarefree_batch(R) == ctx.squarefree_batch(R)


def test_arrangement_resultants_chain(ctx):
    # the projection phase on an arrangement: square-free factorisation of every
    # res(f, f_y) and res(f, g) of five curves (the resultants are the oracle's)
    curves = W.arrangement_curves(8, n=5, d=4, bits=10, conic_frac=0.5, rbits=4)
    rs = [_trim(O.disc_res(f)) for f in curves]
    rs += [_trim(O.res_subres(curves[i], curves[j])) for i in range(5) for j in range(i + 1, 5)]
    rs = [r for r in rs if r]
    got = ctx.squarefree_batch(rs)
    assert got == [_oracle(r) for r in rs]
