"""The seeded input generators against the recipes they state (CPU, small
samples): degree and bit ranges, planted structure (a planted common factor
makes the resultant vanish, the planted gcd factor divides both inputs, the
square-free inputs are the stated products), the shapes of the conic and
arrangement curves, and the serving stream's mix and int64 coefficients."""

import math

import oracle as O
from paper_1103_4697_gb300 import workloads as W


def _tdeg(f):
    return max((j + i for j, r in enumerate(f) for i, c in enumerate(r) if c), default=-1)


def _ydeg(f):
    return max((j for j, r in enumerate(f) if any(r)), default=-1)


def _bits(f):
    return max((abs(int(c)).bit_length() for r in f for c in r), default=0)


def test_mixed_batch_recipe():
    ps = W.mixed_batch(3, n=200)
    planted = sum(ps.planted)
    assert 25 <= planted <= 75                         # a quarter of 200, loosely
    for f, g, p in zip(ps.f, ps.g, ps.planted):
        assert 4 <= len(f) - 1 <= 16 and 4 <= max(len(r) for r in f) - 1 <= 16
        assert len(f) == len(g) and max(len(r) for r in f) == max(len(r) for r in g)   # one box per pair
        if not p:                                      # b-bit signed, b in 8..32: |c| <= 2^(b-1)
            assert 7 <= max(_bits(f), _bits(g)) <= 32
    for f, g, p in list(zip(ps.f, ps.g, ps.planted))[:60]:
        if p:                                          # deg_y h >= 1: the resultant vanishes
            assert O.res_at_prs(f, g, 3) == 0 and O.res_at_prs(f, g, -2) == 0


def test_gcd_batch_recipe():
    P, Q, H = W.gcd_batch(3, n=100)
    for p, q, h in zip(P, Q, H):
        assert 30 <= len(p) - 1 <= 200 and 30 <= len(q) - 1 <= 200
        assert len(h) - 1 == 5 and max(abs(c) for c in h) <= 128
        assert O.divides_z(h, p) and O.divides_z(h, q)


def test_sqf_batch_recipe():
    R, planted = W.sqf_batch(6, n=60)
    for r, (u, facs) in zip(R, planted):
        d1, d2, d3 = (len(x) - 1 for x in facs)
        assert 20 <= d1 <= 60 and 4 <= d2 <= 16 and 0 <= d3 <= 4
        assert 28 <= len(r) - 1 <= 104 and len(r) - 1 == d1 + 2 * d2 + 3 * d3
        assert u != 0 and abs(u) <= 128 and all(max(abs(c) for c in x) <= 1 << 15 for x in facs)
        want = (u,)
        for i, x in enumerate(facs, start=1):
            for _ in range(i):
                want = O.zx_mul(want, tuple(x))
        assert tuple(r) == want


def test_conic_curves_recipe():
    f, g = W.conic_curves(4)
    assert _tdeg(f) == 16 and _ydeg(f) == 16           # 8 conics, and monomials of total degree <= 16
    assert 64 < _bits(f) < 400                          # multi-word coefficients
    assert _tdeg(g) == 24 and _bits(g) <= 64            # dense degree 24, 64-bit


def test_arrangement_curves_recipe():
    cs = W.arrangement_curves(7, n=90)
    conic = [f for f in cs if _bits(f) > 12]
    dense = [f for f in cs if _bits(f) <= 12]
    assert len(cs) == 90 and 10 <= len(conic) <= 40    # a quarter, loosely
    for f in dense:
        assert _tdeg(f) == 8 and _ydeg(f) == 8 and f[8][0] != 0
    for f in conic:
        assert _tdeg(f) == 8 and _bits(f) <= 110
    small = W.arrangement_curves(11, n=1024, d=8, bits=12, conic_frac=0.25, rbits=4)
    assert max(_bits(f) for f in small) <= 57          # the Teissier workload fits int64


def test_serving_stream_recipe():
    reqs = W.serving_stream(5, n=2000, rate=1000.0)
    ts = [r.t_arrive for r in reqs]
    assert ts == sorted(ts) and 1.5 < ts[-1] < 2.6     # 2000 Poisson arrivals at 1000/s
    kinds = sum(r.kind == "res" for r in reqs)
    assert 850 <= kinds <= 1150
    planted = sum(r.planted for r in reqs)
    assert 120 <= planted <= 290
    for r in reqs:
        if r.kind == "res":
            d = max(_tdeg(r.a), _tdeg(r.b))
            coefs = [c for f in (r.a, r.b) for row in f for c in row]
        else:
            d = max(len(r.a), len(r.b)) - 1
            coefs = list(r.a) + list(r.b)
        assert 5 <= d <= 30
        assert all(-(1 << 63) <= c < (1 << 63) for c in coefs)
    # degree draw: round(exp(U(ln 5, ln 30))) puts about half the requests below sqrt(150)
    low = sum(max(len(r.a), len(r.b)) - 1 < math.sqrt(150) for r in reqs if r.kind == "gcd")
    assert 0.35 < low / max(1, len(reqs) - kinds) < 0.65
