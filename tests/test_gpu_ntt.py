"""GPU parity of the root-of-unity point sets (GBR_OPT_POINTS = 2) against the oracle.

With roots of unity the pair is evaluated at the N-th roots of unity modulo each
prime (N the power of two >= max(64, D + 1)) and interpolated by an inverse
number-theoretic transform; the result must be bit-identical to the oracle and
to the integer point sets.  Cases: hand examples and degenerate inputs, the
degree-20 pair (N = 512), the conic product (192 primes, multi-word input),
large x-degree bounds up to the point limit (N = 1024 .. 16384), a mixed batch
(register form and shared-memory evaluation, planted zeros), the per-pair
automatic choice, graph replay, and drop mode (which keeps the integer grid).
"""

import json
import os
import random

import pytest

import oracle as O
from paper_1103_4697_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300.api import Context

    c = Context(device=0, mem_budget=16 << 30)
    c.set_option(N.OPT_POINTS, 2)
    c.set_option(N.OPT_STATS, 1)
    yield c
    c.close()


def _eval(c, a):
    v = 0
    for x in reversed(c):
        v = v * a + x
    return v


def _sparse_long(rng, m, dx, bits):
    """y-degree m, x-degree dx, every coefficient drawn (dense rows in x)."""
    h = 1 << (bits - 1)
    f = [[rng.randint(-h, h - 1) for _ in range(dx + 1)] for _ in range(m + 1)]
    f[-1][-1] = f[-1][-1] or 1
    return f


def test_roots_hand_and_degenerate(ctx):
    gold = json.load(open(os.path.join(HERE, "golden", "hand_examples.json")))
    for e in gold["resultants"]:
        assert ctx.resultant(e["f"], e["g"]) == e["res"]
    f, g = W.small_dense_pair(1)
    assert ctx.resultant(f, g) == list(O.res_bareiss(f, g))
    assert ctx.stats()["root_pairs"] == 1
    for f, g in (([[0]], [[1, 2], [3]]), ([[5]], [[1, 2], [3]]), ([[1, 2], [3]], [[7]]), ([[2]], [[3]])):
        assert ctx.resultant(f, g) == list(O.res_bareiss(f, g)), (f, g)
    for seed, m, n in [(1, 1, 1), (3, 5, 3), (5, 1, 9)]:
        f, g, *_ = W.planted_roots_pair(seed, m, n)
        assert ctx.resultant(f, g) == list(O.res_subres(f, g))


def test_roots_deg20_pair(ctx):
    f, g = W.deg20_pair(2)
    assert ctx.resultant(f, g) == list(O.res_evalz(f, g))
    assert ctx.discriminant_res(f) == list(O.disc_res(f, "evalz"))
    assert ctx.stats()["root_pairs"] == 1


def test_roots_conic_curves(ctx):
    """385 points (N = 512) on 192 primes, multi-word input coefficients."""
    f, g = W.conic_curves(4)
    assert ctx.resultant(f, g) == list(O.res_evalz(f, g))


@pytest.mark.parametrize("m,dx,bits", [(2, 250, 20), (1, 700, 16), (3, 700, 12), (1, 4000, 8), (2, 4095, 8)])
def test_roots_large_point_counts(ctx, m, dx, bits):
    """x-degree bounds D = 2 m dx from 1000 to the point limit (N = 1024 .. 16384):
    every coefficient where the oracle's exact interpolation is quick, else the value
    at four random points; a degree-D polynomial that agrees at a random 32-bit point
    with probability at most D / 2^32."""
    rng = random.Random(m * 100000 + dx)
    f, g = _sparse_long(rng, m, dx, bits), _sparse_long(rng, m, dx, bits)
    r = ctx.resultant(f, g)
    assert ctx.stats()["root_pairs"] == 1
    assert len(r) - 1 <= 2 * m * dx
    if 2 * m * dx <= 1000:
        assert r == list(O.res_evalz(f, g))
    for a in [rng.randint(-2 ** 31, 2 ** 31) for _ in range(4)]:
        assert _eval(r, a) == O.res_at_prs(f, g, a), a


def test_roots_mixed_batch_matches_integer_points(ctx):
    """A heterogeneous batch (register form and shared-memory shapes, y-degrees up to
    40, planted common factors) on roots of unity equals the same batch on integer
    points, and sampled pairs equal the oracle."""
    from paper_1103_4697_gb300 import native as N

    ps = W.mixed_batch(3, 192)
    rng = random.Random(40)
    fs, gs = list(ps.f), list(ps.g)
    for _ in range(6):                          # y-degree 33..40: outside the register form
        m = rng.randint(33, 40)
        fs.append(_sparse_long(rng, m, rng.randint(1, 3), 10))
        gs.append(_sparse_long(rng, rng.randint(m - 3, m), rng.randint(1, 3), 10))
    got = ctx.resultant_batch(fs, gs)
    assert ctx.stats()["root_pairs"] == len(fs)
    ctx.set_option(N.OPT_POINTS, 1)
    try:
        want = ctx.resultant_batch(fs, gs)
        assert ctx.stats()["root_pairs"] == 0
    finally:
        ctx.set_option(N.OPT_POINTS, 2)
    assert got == want
    for q, p in enumerate(ps.planted):
        if p:
            assert got[q] == []
    for q in rng.sample(range(len(fs)), 12):
        a = rng.randint(-2 ** 31, 2 ** 31)
        assert _eval(got[q], a) == O.res_at_prs(fs[q], gs[q], a), q


def test_roots_resident_graph_replay(ctx):
    """A resident batch on roots of unity replayed from its captured graph gives the
    same results as its first run."""
    rng = random.Random(7)
    fs = [_sparse_long(rng, 2, rng.randint(100, 300), 12) for _ in range(24)]
    gs = [_sparse_long(rng, 2, rng.randint(100, 300), 12) for _ in range(24)]
    res = ctx.upload_pairs(fs, gs)
    res.run()
    first = res.fetch()
    res.run()
    assert ctx.stats()["graph_replayed"] == 1
    assert res.fetch() == first
    res.free()
    for q in range(0, 24, 6):
        a = rng.randint(-2 ** 31, 2 ** 31)
        assert _eval(first[q], a) == O.res_at_prs(fs[q], gs[q], a)


def test_automatic_choice_and_drop_mode():
    """GBR_OPT_POINTS = 0 picks roots of unity for pairs whose interpolation dominates
    (small y-degree, large x-degree bound) and integer points for a full tile of
    degree-20 pairs; drop mode keeps the integer grid even when roots are forced;
    results agree."""
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300.api import Context

    rng = random.Random(11)
    long_f = [_sparse_long(rng, 2, 2000, 10) for _ in range(4)]
    long_g = [_sparse_long(rng, 2, 2000, 10) for _ in range(4)]
    F, G = W.deg20_batch_arrays(128)
    with Context(device=0, mem_budget=8 << 30) as c:
        c.set_option(N.OPT_STATS, 1)
        auto_long = c.resultant_batch(long_f, long_g)
        assert c.stats()["root_pairs"] == 4
        auto_d20 = c.resultant_batch(F, G)
        assert c.stats()["root_pairs"] == 0
        c.set_option(N.OPT_POINTS, 1)
        assert c.resultant_batch(long_f, long_g) == auto_long
        c.set_option(N.OPT_POINTS, 2)
        assert c.resultant_batch(F, G) == auto_d20
        assert c.stats()["root_pairs"] == 128
        c.set_option(N.OPT_DROP_UNLUCKY, 1)
        assert c.resultant_batch(F[:2], G[:2]) == auto_d20[:2]
        assert c.stats()["root_pairs"] == 0
        with pytest.raises(Exception):
            c.set_option(N.OPT_POINTS, 4)
