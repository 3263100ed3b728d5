"""GPU parity of the quartic point set (GBR_OPT_POINTS = 3) against the oracle.

The pair is evaluated at 0 and at i^k a (a = 1..h, k = 0..3, i^2 = -1 modulo each
prime); a 4-point transform of the four values at each a gives 4 a^t R_t(a^4) for
the quarter parts of R(x) = sum_t x^t R_t(x^4), and four inverse-Vandermonde
contractions of size about D / 4 give the R_t (half the multiply-adds of the
even/odd split).  The result must be bit-identical to the oracle and to the
symmetric integers.  Cases: hand examples and degenerate inputs, every residue of
the point count modulo 4 (ragged quarter parts), the degree-20 pair, tensor-core
against integer-pipe contractions, point counts above the tensor-core limit up to
the integer-point limit, a mixed batch, the automatic choice, graph replay, and
drop mode (which keeps the integer grid).
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
    c.set_option(N.OPT_POINTS, 3)
    c.set_option(N.OPT_STATS, 1)
    yield c
    c.close()


def _eval(c, a):
    v = 0
    for x in reversed(c):
        v = v * a + x
    return v


def _dense(rng, m, dx, bits):
    h = 1 << (bits - 1)
    f = [[rng.randint(-h, h - 1) for _ in range(dx + 1)] for _ in range(m + 1)]
    f[-1][-1] = f[-1][-1] or 1
    return f


def _with_points(c, mode, fn):
    from paper_1103_4697_gb300 import native as N

    c.set_option(N.OPT_POINTS, mode)
    try:
        return fn()
    finally:
        c.set_option(N.OPT_POINTS, 3)


def test_quad_hand_and_degenerate(ctx):
    gold = json.load(open(os.path.join(HERE, "golden", "hand_examples.json")))
    for e in gold["resultants"]:
        assert ctx.resultant(e["f"], e["g"]) == e["res"]
    f, g = W.small_dense_pair(1)
    assert ctx.resultant(f, g) == list(O.res_bareiss(f, g))
    assert ctx.stats()["quad_pairs"] == 1
    # constant resultants (one point), x-degree bounds 1..3 (quarter parts of 0 or 1
    # coefficient)
    cases = [([[0]], [[1, 2], [3]]), ([[5]], [[1, 2], [3]]), ([[1, 2], [3]], [[7]]), ([[2]], [[3]]),
             ([[1, 1], [1]], [[2], [1]]), ([[1, 1], [1]], [[0, 1], [1]]), ([[0, 1, 1], [1]], [[1, 0, 1], [1]])]
    for f, g in cases:
        assert ctx.resultant(f, g) == list(O.res_bareiss(f, g)), (f, g)
    for seed, m, n in [(1, 1, 1), (3, 5, 3), (5, 1, 9)]:
        f, g, *_ = W.planted_roots_pair(seed, m, n)
        assert ctx.resultant(f, g) == list(O.res_subres(f, g))


def test_quad_every_point_count_mod_4(ctx):
    """Pairs whose x-degree bounds D = 2 m dx cover every residue of P = D + 1 modulo 4
    (R_1 .. R_3 one coefficient shorter than R_0, or not), in groups of one and of
    several pairs with different prime counts: equal to the symmetric integers and to
    the oracle."""
    rng = random.Random(3)
    fs, gs = [], []
    for m, dx in [(1, 1), (1, 2), (2, 1), (1, 3), (3, 1), (2, 2), (1, 5), (5, 1), (3, 2), (2, 3), (4, 3), (3, 5)]:
        for bits in (6, 30):
            fs.append(_dense(rng, m, dx, bits))
            gs.append(_dense(rng, m, rng.randint(0, dx), bits))
    # x-degree bounds D = dx_f n + dx_g m with n != m: odd D too
    for m, n, dxf, dxg in [(2, 3, 1, 2), (3, 2, 2, 1), (1, 4, 3, 1), (4, 1, 1, 2)]:
        fs.append(_dense(rng, m, dxf, 12))
        gs.append(_dense(rng, n, dxg, 12))
    got = ctx.resultant_batch(fs, gs)
    assert ctx.stats()["quad_pairs"] > 0
    want = _with_points(ctx, 1, lambda: ctx.resultant_batch(fs, gs))
    assert got == want
    for f, g, r in zip(fs, gs, got):
        assert r == list(O.res_bareiss(f, g)), (f, g)


def test_quad_deg20_pair(ctx):
    """D = 800: 201 lane pairs, quarter parts of 201 and 200 coefficients."""
    f, g = W.deg20_pair(2)
    assert ctx.resultant(f, g) == list(O.res_evalz(f, g))
    assert ctx.stats()["quad_pairs"] == 1
    assert ctx.discriminant_res(f) == list(O.disc_res(f, "evalz"))


def test_quad_tensor_cores_match_integer_pipes(ctx):
    """Quarter contractions up to 256 points on the tensor cores, larger ones on the
    integer pipes: 150 pairs sharing one point count (two pair tiles) and counts on
    both sides of the limit in one batch; equal with the tensor cores off and equal
    to the oracle."""
    from paper_1103_4697_gb300.native import OPT_INTERP_TC

    fs, gs = [], []
    for i in range(150):
        f, g = W.small_dense_pair(900 + i, 4, 12)
        fs.append(f)
        gs.append(g)
    for d, bits in ((3, 30), (7, 20), (10, 16), (15, 8), (16, 8), (23, 6), (31, 4)):
        f, g = W.small_dense_pair(950 + d, d, bits)
        fs.append(f)
        gs.append(g)
    got = ctx.resultant_batch(fs, gs)
    assert ctx.stats()["quad_pairs"] == len(fs)
    ctx.set_option(OPT_INTERP_TC, 0)
    try:
        ref = ctx.resultant_batch(fs, gs)
    finally:
        ctx.set_option(OPT_INTERP_TC, 1)
    assert got == ref
    for q in (0, 77, 149, 150, 151):
        assert got[q] == list(O.res_bareiss(fs[q], gs[q]))
    rng = random.Random(11)
    for q in range(152, len(fs)):
        for a in (rng.randint(-10 ** 6, 10 ** 6), rng.randint(-10 ** 6, 10 ** 6)):
            assert _eval(got[q], a) == O.res_at_prs(fs[q], gs[q], a)


@pytest.mark.parametrize("m,dx,bits", [(1, 510, 16), (2, 256, 12), (1, 1000, 10), (2, 1024, 8)])
def test_quad_large_point_counts(ctx, m, dx, bits):
    """x-degree bounds D = 2 m dx from 1020 to the integer-point limit 4096 (quarter
    matrices of 256 to 1025 points: the tensor-core limit and beyond): values at four
    random points, each a degree-D polynomial identity that a wrong result passes with
    probability at most D / 2^32."""
    rng = random.Random(m * 100000 + dx)
    f, g = _dense(rng, m, dx, bits), _dense(rng, m, dx, bits)
    r = ctx.resultant(f, g)
    assert ctx.stats()["quad_pairs"] == 1
    assert len(r) - 1 <= 2 * m * dx
    for a in [rng.randint(-2 ** 31, 2 ** 31) for _ in range(4)]:
        assert _eval(r, a) == O.res_at_prs(f, g, a), a


def test_quad_mixed_batch_matches_integer_points(ctx):
    """A heterogeneous batch (register form and shared-memory shapes, planted common
    factors, y-degrees up to 40) on the quartic set equals the same batch on the
    symmetric integers, and sampled pairs equal the oracle."""
    ps = W.mixed_batch(3, 192)
    rng = random.Random(40)
    fs, gs = list(ps.f), list(ps.g)
    for _ in range(6):
        m = rng.randint(33, 40)
        fs.append(_dense(rng, m, rng.randint(1, 3), 10))
        gs.append(_dense(rng, rng.randint(m - 3, m), rng.randint(1, 3), 10))
    got = ctx.resultant_batch(fs, gs)
    assert ctx.stats()["quad_pairs"] > 0
    want = _with_points(ctx, 1, lambda: ctx.resultant_batch(fs, gs))
    assert got == want
    for q, p in enumerate(ps.planted):
        if p:
            assert got[q] == []
    for q in rng.sample(range(len(fs)), 12):
        a = rng.randint(-2 ** 31, 2 ** 31)
        assert _eval(got[q], a) == O.res_at_prs(fs[q], gs[q], a), q


def test_quad_deg20_batch_and_graph_replay(ctx):
    """512 degree-20 pairs as a resident batch: the first run, the stage-graph replay
    and the whole-step graph replay give the symmetric integers' results."""
    F, G = W.deg20_batch_arrays(512)
    want = _with_points(ctx, 1, lambda: ctx.resultant_batch(F, G))
    assert ctx.resultant_batch(F, G) == want
    assert ctx.stats()["quad_pairs"] == 512
    res = ctx.upload_pairs(F, G)
    seen = set()
    for _ in range(5):
        res.run()
        seen.add(ctx.stats()["graph_replayed"])
        assert res.fetch() == want
    res.free()
    assert 2 in seen
    for q in (0, 255, 511):
        assert want[q] == list(O.res_evalz(F[q], G[q]))


def test_quad_automatic_choice_and_drop_mode():
    """GBR_OPT_POINTS = 0 takes the quartic set for a full tile of degree-20 pairs and
    roots of unity for long low-degree pairs; drop mode keeps the integer grid when
    the quartic set is forced; results agree."""
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300.api import Context

    F, G = W.deg20_batch_arrays(128)
    with Context(device=0, mem_budget=8 << 30) as c:
        c.set_option(N.OPT_STATS, 1)
        auto = c.resultant_batch(F, G)
        st = c.stats()
        assert st["quad_pairs"] == 128 and st["root_pairs"] == 0
        c.set_option(N.OPT_POINTS, 1)
        assert c.resultant_batch(F, G) == auto
        assert c.stats()["quad_pairs"] == 0
        c.set_option(N.OPT_POINTS, 3)
        c.set_option(N.OPT_DROP_UNLUCKY, 1)
        assert c.resultant_batch(F[:2], G[:2]) == auto[:2]
        assert c.stats()["quad_pairs"] == 0
