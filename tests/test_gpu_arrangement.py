"""GPU parity: the resultants of a curve arrangement (Section 3, curve-pair
analysis: R_C = res(f_C, f_C,y) for every curve, R_CD = res(f_C, f_D) for every
pair) from one device pass equal the CPU oracle exactly, job by job.
"""

import numpy as np
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


def _trim(a):
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def _check(curves, disc, pairs, var=1):
    cs = curves if var == 1 else [np.array(f, dtype=object).T.tolist() for f in curves]
    for i, f in enumerate(cs):
        assert disc[i] == _trim(O.disc_res(f)), i
    for (i, j), r in pairs.items():
        assert r == _trim(O.res_subres(cs[i], cs[j])), (i, j)


@pytest.mark.parametrize("seed,n,d", [(1, 5, 3), (2, 7, 4), (3, 4, 6)])
def test_arrangement_matches_oracle(ctx, seed, n, d):
    curves = W.arrangement_curves(seed, n=n, d=d, bits=10, conic_frac=0.5, rbits=4)
    disc, pairs = ctx.arrangement_resultants(curves)
    assert len(disc) == n and len(pairs) == n * (n - 1) // 2
    _check(curves, disc, pairs)


def test_arrangement_eliminating_x(ctx):
    curves = W.arrangement_curves(4, n=4, d=4, bits=8, conic_frac=0.5, rbits=3)
    disc, pairs = ctx.arrangement_resultants(curves, var=0)
    _check(curves, disc, pairs, var=0)


def test_degenerate_sizes(ctx):
    assert ctx.arrangement_resultants([]) == ([], {})
    f = [[-25, 0, 1], [0, 0, 0], [1, 0, 0]]          # circle x^2 + y^2 = 25
    disc, pairs = ctx.arrangement_resultants([f])
    assert pairs == {} and disc == [_trim(O.disc_res(f))]
    # a curve without y (a vertical-line pencil), a constant, a repeated curve
    g = [[-4, 0, 1]]
    h = [[3]]
    curves = [f, g, h, f]
    disc, pairs = ctx.arrangement_resultants(curves)
    _check(curves, disc, pairs)
    assert pairs[(0, 3)] == []                        # a curve and itself: res = 0


def test_mixed_widths_and_shared_uploads(ctx):
    # one curve with coefficients wider than 64 bits next to small ones
    big = [[2**70 + 1, 3, -(2**66)], [5, -7, 0], [1, 0, 0]]
    curves = W.arrangement_curves(5, n=3, d=3, bits=12, conic_frac=0.0) + [big]
    disc, pairs = ctx.arrangement_resultants(curves)
    _check(curves, disc, pairs)


def test_resident_arrangement_replays(ctx):
    curves = W.arrangement_curves(6, n=9, d=5, bits=12, conic_frac=0.3, rbits=5)
    disc, pairs = ctx.arrangement_resultants(curves)
    want = disc + [pairs[(i, j)] for i in range(9) for j in range(i + 1, 9)]
    res = ctx.upload_arrangement(curves)
    try:
        for _ in range(3):                            # plain run, capture, replay
            res.run()
            assert res.fetch() == want
    finally:
        res.free()
    # spot-check against the oracle
    for q, (i, j) in enumerate([(0, 1), (3, 8), (7, 8)]):
        assert pairs[(i, j)] == _trim(O.res_subres(curves[i], curves[j]))
    assert disc[4] == _trim(O.disc_res(curves[4]))
