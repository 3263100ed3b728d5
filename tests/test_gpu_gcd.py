"""GPU parity: gcd(p, q) in Z[x] from libgbres equals the CPU oracle exactly."""

import json
import math
import os
import random

import pytest

import oracle as O
from paper_1103_4697_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    from paper_1103_4697_gb300.api import Context

    c = Context(device=0, mem_budget=8 << 30)
    yield c
    c.close()


def test_hand_examples(ctx):
    gold = json.load(open(os.path.join(HERE, "golden", "hand_examples.json")))
    for e in gold["gcds"]:
        p, q = e["p"] or [0], e["q"] or [0]
        assert ctx.gcd(p, q) == e["gcd"], e


def test_small_pair_gcd(ctx):
    f, g = W.small_dense_pair(1)
    p, q = list(f[0]), list(g[0])        # f(x, 0), g(x, 0)
    assert ctx.gcd(p, q) == list(O.gcd_z(p, q))


def test_planted_factor_batch(ctx):
    P, Q, H = W.gcd_batch(21, 97, lo=10, hi=60, hdeg=5)
    out = ctx.gcd_batch(P, Q)
    for p, q, h, g in zip(P, Q, H, out):
        assert g == list(O.gcd_z(p, q))
        assert O.divides_z(h, g)


def test_contents_signs_constants(ctx):
    rng = random.Random(4)
    cases = [
        ([6, 12, 6], [4, 4]),                     # 6(x+1)^2, 4(x+1)
        ([-3, 0, 3], [5, 5]),                     # negative coefficients, content 3 and 5
        ([7], [14, 21]),                          # constant
        ([0, 0, 0, 5], [0, 0, 10]),               # x^3 and x^2 (gcd x^2 times content gcd 5)
        ([2, -4], [0]),                           # q = 0
        ([0], [-6, 3, 9]),                        # p = 0, negative leading coefficient flips
        ([1, 1], [1, -1]),                        # coprime
        ([-2 ** 62, 2 ** 62], [2 ** 61, 2 ** 61]),   # large contents
    ]
    for p, q in cases:
        assert ctx.gcd(p, q) == list(O.gcd_z(p, q)), (p, q)
    for _ in range(20):
        h = [rng.randint(-9, 9) for _ in range(rng.randint(1, 4))]
        h[-1] = h[-1] or -3
        u = [rng.randint(-99, 99) for _ in range(rng.randint(1, 12))]
        v = [rng.randint(-99, 99) for _ in range(rng.randint(1, 12))]
        u[-1] = u[-1] or 1
        v[-1] = v[-1] or 1
        p = list(O.zx_mul(tuple(rng.choice([1, 2, 6]) * c for c in h), tuple(u)))
        q = list(O.zx_mul(tuple(rng.choice([1, 3, -4]) * c for c in h), tuple(v)))
        assert ctx.gcd(p, q) == list(O.gcd_z(p, q)), (p, q)


def test_unlucky_and_lc_divisible_primes(ctx):
    """mod p0 and p1 the linear factors x + a and x + a + p0 p1 coincide, so those
    primes see a spurious common factor and must be outvoted by the degree rule;
    lc(P) = p2 makes p2 unusable."""
    from paper_1103_4697_gb300.api import primes

    p0, p1, p2 = primes(3)
    a = 12345
    P = list(O.zx_mul((a, 1), (1, 1, 1)))
    Q = list(O.zx_mul((a + p0 * p1, 1), (2, 0, 1)))
    assert ctx.gcd(P, Q) == list(O.gcd_z(P, Q)) == [1]
    h = (3, -1, 2)
    P2 = list(O.zx_mul(h, (5, p2)))
    Q2 = list(O.zx_mul(h, (7, 1, 1)))
    assert ctx.gcd(P2, Q2) == list(O.gcd_z(P2, Q2))


def _coprime_mod(a, b, p=1_000_000_007):
    """True when a and b are coprime modulo p with p not dividing either leading
    coefficient; this proves them coprime over Q (a common factor over Z would
    survive reduction mod p with its degree)."""
    a = [x % p for x in a]
    b = [x % p for x in b]
    if a[-1] == 0 or b[-1] == 0:
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


def test_large_degree(ctx):
    """Degree 600..800 inputs (several shared-memory tiles per warp)."""
    P, Q, H = W.gcd_batch(33, 2, lo=600, hi=800, hdeg=7)
    out = ctx.gcd_batch(P, Q)
    for p, q, h, g in zip(P, Q, H, out):
        assert g and g[-1] > 0
        assert O.divides_z(h, g)
        assert O.divides_z(g, p) and O.divides_z(g, q)
        cp, cq = O.zx_divexact(tuple(p), tuple(g)), O.zx_divexact(tuple(q), tuple(g))
        assert _coprime_mod(list(cp), list(cq))
        assert O.content(g) == math.gcd(O.content(p), O.content(q))


def test_gcd_batch_every_job(ctx):
    """4096 jobs, degrees 30..200, planted degree-5 factor: every job checked by the
    defining properties of the gcd over Z (divides both inputs, coprime cofactors,
    content, sign) and the planted factor divides it; 512 jobs equal the oracle's gcd."""
    import oracle_tasks as T

    P, Q, H = W.gcd_batch(3, 4096)
    out = ctx.gcd_batch(P, Q)
    for i in range(4096):
        assert O.divides_z(H[i], out[i]), i
    rng = random.Random(9)
    exact = rng.sample(range(4096), 512)
    with T.pool() as pool:
        ok = pool.map(T.gcd_is_gcd, [(P[i], Q[i], out[i]) for i in range(4096)], chunksize=32)
        want = pool.map(T.gcd_exact, [(P[i], Q[i]) for i in exact], chunksize=4)
    assert all(ok), [i for i in range(4096) if not ok[i]][:10]
    for i, w in zip(exact, want):
        assert out[i] == w, i


def test_mixed_batch_equals_separate_calls(ctx):
    """gbr_mixed_batch (the gcd half on a worker stream beside the resultant half) gives
    exactly what gbr_resultant_batch and gbr_gcd_batch give: the heterogeneous resultant
    batch at its full 4096 pairs (pipelined over the context's workers) with the 4096
    gcd jobs; planted pairs give 0; either half may be empty."""
    ps = W.mixed_batch(3, 4096)
    P, Q, H = W.gcd_batch(3, 4096)
    res, gcds = ctx.mixed_batch(ps.f, ps.g, P, Q)
    assert res == ctx.resultant_batch(ps.f, ps.g)
    assert gcds == ctx.gcd_batch(P, Q)
    assert all(res[i] == [] for i in range(4096) if ps.planted[i])
    for i in range(0, 4096, 1024):
        assert gcds[i] == list(O.gcd_z(P[i], Q[i]))
    r2, g2 = ctx.mixed_batch([], [], P[:3], Q[:3])
    assert r2 == [] and g2 == gcds[:3]
    r3, g3 = ctx.mixed_batch(ps.f[:5], ps.g[:5], [], [])
    assert r3 == res[:5] and g3 == []
