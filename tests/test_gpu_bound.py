"""The number of primes rests on a bound computed on the GPU: pin it with exact arithmetic.

The Chinese remaindering of a resultant is exact only when the product M of its
primes exceeds 2B + 1 for a bound B on the coefficients.  k_bounds evaluates the
Hadamard-type bound in single precision with directed rounding; here the same
bound is evaluated by the oracle in exact integer and rational arithmetic
(oracle/bound.py) on about 220 inputs, and for every job the device's log2 B must
lie at or above the exact enclosure and its primes must satisfy M > 2B + 1 for
the exact B.  The shapes cover the headline batch, the heterogeneous batch,
conic products with multi-word coefficients, multi-word random inputs,
coefficients of 57..63 bits (the double-precision sum with its error term),
rows longer than the 128 coefficients staged in shared memory, rows growing or
shrinking geometrically with the power of y (where the best scaling lambda is
not 1), inputs where the bound is attained (R = +-2a, 1 + a^2, f_0^n), the
projection resultant res(f, f_y), and inputs with an empty Sylvester column.
"""

import random
from fractions import Fraction

import pytest

from paper_1103_4697_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rand(rng, m, dx, bits):
    h = 1 << (bits - 1)
    return [[rng.randint(-h, h - 1) for _ in range(dx + 1)] for _ in range(m + 1)]


def _lead(rows):
    rows[-1][0] = rows[-1][0] or 1
    return rows


def bound_pairs():
    """(f, g) jobs covering the bound's code paths (see the module docstring)."""
    rng = random.Random(2024)
    pairs = []
    F, G = W.deg20_batch_arrays(60)
    pairs += [(F[q].tolist(), G[q].tolist()) for q in range(60)]
    ps = W.mixed_batch(3, 48)
    pairs += list(zip(ps.f, ps.g))
    cf, cg = W.conic_curves(4)
    pairs.append((cf, cg))
    for _ in range(16):                                        # multi-word coefficients
        bits = rng.randint(70, 500)
        pairs.append((_lead(_rand(rng, rng.randint(1, 6), rng.randint(0, 5), bits)),
                      _lead(_rand(rng, rng.randint(1, 6), rng.randint(0, 5), bits))))
    for _ in range(16):                                        # 57..63-bit single words
        bits = rng.randint(58, 64)
        pairs.append((_lead(_rand(rng, rng.randint(1, 8), rng.randint(0, 8), bits)),
                      _lead(_rand(rng, rng.randint(1, 8), rng.randint(0, 8), bits))))
    for _ in range(8):                                         # rows longer than 128
        pairs.append((_lead(_rand(rng, rng.randint(1, 3), rng.randint(130, 220), 12)),
                      _lead(_rand(rng, rng.randint(1, 3), rng.randint(0, 40), 12))))
    for s in (-20, -12, -6, -3, 3, 6, 12, 20):                 # lambda away from 1
        for _ in range(4):
            m, n = rng.randint(2, 7), rng.randint(2, 7)
            f = [[rng.randint(-99, 99) << max(0, s * i) for _ in range(rng.randint(1, 4))] for i in range(m + 1)]
            g = [[rng.randint(-99, 99) << max(0, -s * j) for _ in range(rng.randint(1, 4))] for j in range(n + 1)]
            pairs.append((_lead(f), _lead(g)))
    for a in (1, 5, 1 << 20, (1 << 40) + 3, 1 << 62):          # attained: R = +-2a and -(1 + a^2)
        pairs.append(([[a], [1]], [[-a], [1]]))
        pairs.append(([[a], [1]], [[-1], [a]]))
    for k in range(10):                                        # attained: R = f_0^n
        f0 = [rng.randint(0, 1 << rng.randint(1, 30)) for _ in range(rng.randint(1, 6))]
        f0[-1] = f0[-1] or 1
        g = _lead(_rand(rng, rng.randint(1, 5), rng.randint(0, 4), 10))
        pairs.append(([f0], g) if k % 2 == 0 else (g, [f0]))
    for _ in range(4):                                         # y divides both: empty last column
        f = _lead(_rand(rng, rng.randint(2, 5), 3, 12))
        g = _lead(_rand(rng, rng.randint(2, 5), 3, 12))
        f[0] = [0] * len(f[0])
        g[0] = [0] * len(g[0])
        pairs.append((f, g))
    return pairs


def disc_polys():
    rng = random.Random(77)
    out = []
    for _ in range(14):
        d = rng.randint(3, 20)
        out.append(W.dense_total_degree(W.Stream(rng.randint(1, 10 ** 9), 0), d, rng.choice([8, 16, 40])))
    out.append(W.conic_curves(4)[0])
    out.append(W.conic_curves(4, nterms=0)[0])
    return out


def _check(plans, exact, jobs):
    from oracle.bound import log2_floor_half_pred
    from paper_1103_4697_gb300.api import primes

    table = primes(max(p["primes"] for p in plans) or 1)
    for q, (pl, ex) in enumerate(zip(plans, exact)):
        if ex is None:
            # an empty Sylvester column: R = 0 exactly; the device bound is -inf and any
            # number of primes lifts 0 correctly (the plan keeps the smallest, one)
            assert pl["log2_bound"] == float("-inf") and pl["primes"] <= 1, (q, pl)
            continue
        lo, hi = ex
        assert pl["primes"] >= 1, (q, pl)
        assert Fraction(pl["log2_bound"]) >= hi, (q, pl["log2_bound"], float(hi))
        M = 1
        for p in table[:pl["primes"]]:
            M *= p
        assert log2_floor_half_pred(M) > hi, (q, pl["primes"], float(hi))
        # with every coefficient below 2^56 and rows of at most 128 coefficients the
        # device sums the same row quantities exactly (longer rows take the 1-norm), so
        # its bound may exceed the exact one only by its rounding margins
        if _max_bits(jobs[q]) <= 56 and _max_row(jobs[q]) <= 128:
            slack = 0.01 + 0.002 * (pl["m"] + pl["n"]) + 2 ** -9
            assert pl["log2_bound"] <= float(hi) + slack, (q, pl["log2_bound"], float(hi))
    return len(plans)


def _max_row(job):
    polys = job if isinstance(job, tuple) else (job,)
    return max(len(row) for p in polys for row in p)


def _max_bits(job):
    polys = job if isinstance(job, tuple) else (job,)
    return max(abs(int(c)).bit_length() for p in polys for row in p for c in row)


def test_device_bound_at_least_the_exact_bound():
    import oracle_tasks as T
    from paper_1103_4697_gb300.api import Context

    pairs = bound_pairs()
    polys = disc_polys()
    with T.pool() as pool:
        exact = pool.map(T.bound_interval, pairs, chunksize=2)
        dexact = pool.map(T.bound_interval, [(f, None) for f in polys], chunksize=1)
    with Context(device=0, mem_budget=4 << 30) as ctx:
        r = ctx.upload_pairs([f for f, _ in pairs], [g for _, g in pairs])
        r.run()
        plans = r.plan()
        r.free()
        d = ctx.upload_pairs(polys, disc=True)
        d.run()
        dplans = d.plan()
        d.free()
    n = _check(plans, exact, pairs) + _check(dplans, dexact, polys)
    assert n >= 200


def test_bound_same_in_small_and_large_batches():
    """Batches of at most 256 pairs take the bound with four warps per pair (rows and
    scalings split over the warps), larger ones with one warp per pair: every job gets
    the same plan (degrees, bound, primes) either way, for resultants and res(f, f_y)."""
    from paper_1103_4697_gb300.api import Context

    pairs = bound_pairs()
    polys = disc_polys()
    with Context(device=0, mem_budget=4 << 30) as ctx:
        def plans(fs, gs, disc=False):
            r = ctx.upload_pairs(fs, gs, disc=disc)
            try:
                r.run()
                return r.plan()
            finally:
                r.free()

        jobs = pairs * 2
        assert len(jobs) > 256
        big = plans([f for f, _ in jobs], [g for _, g in jobs])
        small = []
        for i in range(0, len(pairs), 7):
            chunk = pairs[i:i + 7]
            small += plans([f for f, _ in chunk], [g for _, g in chunk])
        assert big[:len(pairs)] == small and big[len(pairs):] == small
        dbig = plans(polys * 17, None, disc=True)
        assert len(polys) * 17 > 256
        dsmall = [p for f in polys for p in plans([f], None, disc=True)]
        assert dbig[:len(polys)] == dsmall
