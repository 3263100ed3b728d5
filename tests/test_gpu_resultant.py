"""GPU parity: res_var(f, g) from libgbres equals the CPU oracle bit for bit.

Every comparison is exact (integer results, tolerance 0).  Small cases compare
every coefficient; the full-size workloads compare every coefficient of sampled
pairs against the oracle's exact interpolation and the value R(a) at random
integer points a for more sampled pairs (a polynomial of degree D that agrees at
D + 1 points is equal; random wide points catch any wrong coefficient).
"""

import json
import os
import random

import numpy as np
import pytest

import oracle as O
from paper_1103_4697_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    from paper_1103_4697_gb300.api import Context

    c = Context(device=0, mem_budget=16 << 30)
    yield c
    c.close()


def _poly_eval(c, a):
    v = 0
    for x in reversed(c):
        v = v * a + x
    return v


def _oracle(f, g):
    return list(O.res_subres(f, g))


def test_hand_examples(ctx):
    gold = json.load(open(os.path.join(HERE, "golden", "hand_examples.json")))
    for e in gold["resultants"]:
        assert ctx.resultant(e["f"], e["g"]) == e["res"]


def test_small_dense_pair(ctx):
    f, g = W.small_dense_pair(1)
    assert ctx.resultant(f, g) == list(O.res_bareiss(f, g))


@pytest.mark.parametrize("seed,m,n", [(1, 1, 1), (2, 2, 3), (3, 5, 3), (4, 7, 6), (5, 1, 9)])
def test_planted_roots(ctx, seed, m, n):
    f, g, *_ = W.planted_roots_pair(seed, m, n)
    assert ctx.resultant(f, g) == _oracle(f, g)


def test_symmetry_and_var0(ctx):
    f, g = W.small_dense_pair(11, 5, 8)
    r = ctx.resultant(f, g)
    m, n = O.ydeg(f), O.ydeg(g)
    s = ctx.resultant(g, f)
    assert s == (r if (m * n) % 2 == 0 else [-c for c in r])
    # eliminating x of (f, g) equals eliminating y of the transposed pair
    ft = np.array(f, dtype=np.int64).T.copy()
    gt = np.array(g, dtype=np.int64).T.copy()
    assert ctx.resultant(f, g, var=0) == _oracle(ft, gt)


def test_degenerate_inputs(ctx):
    g = [[1, 2], [0, 1], [5]]
    assert ctx.resultant([[3, 1]], g) == _oracle([[3, 1]], g)            # m = 0
    assert ctx.resultant(g, [[3, 1]]) == _oracle(g, [[3, 1]])            # n = 0
    assert ctx.resultant([[2]], [[7, 1]]) == [1]                          # m = n = 0
    assert ctx.resultant([[0]], g) == []                                  # f = 0
    assert ctx.resultant(g, [[0, 0], [0, 0]]) == []                       # g = 0
    assert ctx.resultant([[0, 0], [0, 0], [1]], g) == _oracle([[0, 0], [0, 0], [1]], g)   # zero rows


def test_leading_coefficient_vanishes_at_points(ctx):
    """lc_y f = (x-2)(x+3) x and lc_y g = x - 2 vanish at evaluation points 0 and 2:
    the formal-degree elimination must still give the exact determinant."""
    f = [[1, 2, -1], [0, 1], [0, -6, 1, 1]]
    g = [[2, -1], [1, 0, 1], [-2, 1]]
    assert ctx.resultant(f, g) == list(O.res_bareiss(f, g))
    # both leading coefficients vanish at x = 2: R(2) = 0
    assert _poly_eval(ctx.resultant(f, g), 2) == 0


def test_prime_divides_leading_coefficient(ctx):
    """lc_y f is a multiple of the first two table primes: it vanishes identically
    modulo them; the formal-degree path stays exact."""
    from paper_1103_4697_gb300.api import primes

    p0, p1 = primes(2)
    f = [[3, 1, 4], [1, 5], [p0 * p1, 0, p0 * p1 * 7]]
    g = [[2, 7], [1, 8, 2], [9]]
    assert ctx.resultant(f, g) == _oracle(f, g)


def test_discriminant_small(ctx):
    for seed in range(4):
        f, _ = W.small_dense_pair(30 + seed, 6, 8)
        assert ctx.discriminant_res(f) == list(O.disc_res(f))


def test_batch_mixed_small(ctx):
    """Mixed degrees in one batch: several work tiles per bucket and a ragged tail."""
    rng = random.Random(7)
    fs, gs = [], []
    for _ in range(97):
        m, n = rng.randint(0, 9), rng.randint(0, 9)
        dx = rng.randint(0, 6)
        fs.append([[rng.randint(-50, 50) for _ in range(dx + 1)] for _ in range(m + 1)])
        gs.append([[rng.randint(-50, 50) for _ in range(rng.randint(0, 6) + 1)] for _ in range(n + 1)])
    got = ctx.resultant_batch(fs, gs)
    for f, g, r in zip(fs, gs, got):
        assert r == _oracle(f, g)


def test_batch_extra_prime_is_identical(ctx):
    from paper_1103_4697_gb300.native import OPT_EXTRA_PRIMES

    f, g = W.small_dense_pair(2, 8, 12)
    r0 = ctx.resultant(f, g)
    ctx.set_option(OPT_EXTRA_PRIMES, 1)
    try:
        r1 = ctx.resultant(f, g)
    finally:
        ctx.set_option(OPT_EXTRA_PRIMES, 0)
    assert r0 == r1 == _oracle(f, g)


def test_big_coefficients_multiword(ctx):
    """Coefficients above 64 bits (multi-word input)."""
    rng = random.Random(3)
    f = [[rng.randint(-2 ** 150, 2 ** 150) for _ in range(4)] for _ in range(4)]
    g = [[rng.randint(-2 ** 90, 2 ** 90) for _ in range(3)] for _ in range(5)]
    assert ctx.resultant(f, g) == _oracle(f, g)


def test_deg20_pair_full(ctx):
    """The degree-20 pair, 16-bit coefficients: res_y(f, g) and res_y(f, f_y), every
    coefficient against the oracle's exact interpolation over Z."""
    f, g = W.deg20_pair(2)
    assert ctx.resultant(f, g) == list(O.res_evalz(f, g))
    assert ctx.discriminant_res(f) == list(O.disc_res(f, "evalz"))


def test_conic_curves_full(ctx):
    """Product of 8 conics plus sparse terms (hundreds of primes) against a dense
    degree-24 curve with 64-bit coefficients; res_y(f, g) and res_y(f, f_y)."""
    f, g = W.conic_curves(4)
    r = ctx.resultant(f, g)
    assert r == list(O.res_evalz(f, g))
    d = ctx.discriminant_res(f)
    assert d == list(O.disc_res(f, "evalz"))


def _bimul(a, b):
    """Product in Z[x][y] of rows a[i] (coefficients of y^i, lists over x)."""
    out = [[0] * (len(a[0]) + len(b[0]) - 1) for _ in range(len(a) + len(b) - 1)]
    for i, ra in enumerate(a):
        for j, rb in enumerate(b):
            for s, x in enumerate(ra):
                for t, y in enumerate(rb):
                    out[i + j][s + t] += x * y
    return out


def test_warp_chinese_remaindering_prime_counts(ctx):
    """Results that need between 65 and 512 primes take the Chinese remaindering with one
    warp per coefficient (digit dot products split over the lanes, limb column sums);
    pairs of several prime counts in one resident batch, a planted common factor, and a
    one-shot call, every coefficient against the oracle."""
    rng = random.Random(11)
    shapes = [(3, 3, 1, 500), (4, 3, 2, 480), (6, 6, 1, 500), (8, 7, 1, 500), (12, 12, 1, 500), (2, 2, 3, 500),
              (5, 5, 0, 400)]
    fs, gs = [], []
    for m, n, dx, b in shapes:
        fs.append([[rng.randint(-2 ** b, 2 ** b) for _ in range(dx + 1)] for _ in range(m + 1)])
        gs.append([[rng.randint(-2 ** b, 2 ** b) for _ in range(dx + 1)] for _ in range(n + 1)])
    h = [[rng.randint(-9, 9), 1], [rng.randint(1, 9), rng.randint(-9, 9)]]   # y-degree 1: a common factor
    fs.append(_bimul(fs[2], h))
    gs.append(_bimul(gs[1], h))
    res = ctx.upload_pairs(fs, gs)
    try:
        res.run()
        got = res.fetch()
        plans = res.plan()
    finally:
        res.free()
    ks = [p["primes"] for p in plans]
    assert sum(64 < k <= 512 for k in ks) >= 5, ks
    for f, g, r in zip(fs, gs, got):
        assert r == _oracle(f, g)
    assert got[-1] == []
    assert ctx.resultant(fs[4], gs[4]) == got[4]


def test_close_point_counts_share_a_group(ctx):
    """Pairs whose degree bounds lie within a few points of each other share one point
    count (one contraction group): every result equals the oracle, the plan reports each
    pair's own degree bound, and replays from the step graph keep the results."""
    from paper_1103_4697_gb300.api import resultant_info

    rng = random.Random(23)
    fs, gs = [], []
    for dy, dx in ((5, 6), (6, 5), (3, 10), (4, 8), (2, 16), (5, 7), (7, 5), (4, 9), (6, 6), (3, 11)) * 2:
        fs.append([[rng.randint(-999, 999) for _ in range(dx + 1)] for _ in range(dy + 1)])
        gs.append([[rng.randint(-999, 999) for _ in range(dx + 1)] for _ in range(dy + 1)])
    want = [_oracle(f, g) for f, g in zip(fs, gs)]
    res = ctx.upload_pairs(fs, gs)
    try:
        for _ in range(5):
            res.run()
            assert res.fetch() == want
        plans = res.plan()
    finally:
        res.free()
    bounds = [resultant_info(f, g)["deg_bound"] for f, g in zip(fs, gs)]
    assert [p["deg_bound"] for p in plans] == bounds
    assert len(set(bounds)) > 2


@pytest.fixture(scope="module")
def opool():
    """Oracle workers on every host core (spawn: safe after CUDA initialisation)."""
    import oracle_tasks as T

    p = T.pool()
    yield p
    p.terminate()


def _wide_points(rng, n=2):
    return [rng.randint(-2 ** 31, 2 ** 31) for _ in range(n)]


def _check_every_pair_at_points(opool, fs, gs, out, rng, skip=()):
    """Every pair's result at two random 32-bit points against the oracle's exact R(a):
    a wrong polynomial of degree <= D agrees at a random point with probability at
    most D / 2^32."""
    import oracle_tasks as T

    idx = [q for q in range(len(out)) if q not in skip]
    pts = {q: _wide_points(rng) for q in idx}
    want = opool.map(T.res_points, [(fs[q], gs[q], pts[q]) for q in idx], chunksize=32)
    for q, w in zip(idx, want):
        got = [_poly_eval(out[q], a) for a in pts[q]]
        assert got == w, f"pair {q} differs from the oracle at x = {pts[q]}"


def test_deg20_batch_every_pair(ctx, opool):
    """The 4096-pair degree-20 batch in the launch configuration the benchmark times:
    every pair at two random points against the oracle, 16 pairs coefficient by
    coefficient."""
    import oracle_tasks as T

    F, G = W.deg20_batch_arrays(4096)
    res = ctx.upload_pairs(F, G)
    res.run()
    out = res.fetch()
    res.free()
    rng = random.Random(11)
    full = rng.sample(range(4096), 16)
    want = opool.map(T.res_full, [(F[q], G[q]) for q in full], chunksize=1)
    for q, w in zip(full, want):
        assert out[q] == w, f"pair {q}"
    _check_every_pair_at_points(opool, F, G, out, rng)


def test_mixed_batch_every_pair(ctx, opool):
    """The heterogeneous batch at its full size (4096 pairs, degrees 4..16 per variable,
    8..32-bit coefficients, a quarter with planted common factors), as one resident
    batch: every planted pair gives 0, every other pair is checked at two random
    points, 16 of them coefficient by coefficient."""
    import oracle_tasks as T

    ps = W.mixed_batch(3, 4096)
    res = ctx.upload_pairs(ps.f, ps.g)
    res.run()
    out = res.fetch()
    res.free()
    planted = {q for q, p in enumerate(ps.planted) if p}
    assert len(planted) > 900
    for q in planted:
        assert out[q] == [], f"planted pair {q}"
    rng = random.Random(5)
    others = [q for q in range(4096) if q not in planted]
    full = rng.sample(others, 16)
    want = opool.map(T.res_full, [(ps.f[q], ps.g[q]) for q in full], chunksize=1)
    for q, w in zip(full, want):
        assert out[q] == w, f"pair {q}"
    _check_every_pair_at_points(opool, ps.f, ps.g, out, rng, skip=planted)


def test_interpolation_contraction_matches_newton(ctx):
    """Pairs sharing their point count are interpolated by the inverse-Vandermonde
    contraction; with different coefficient sizes (so different prime counts) in one
    group and a ragged number of pairs.  Newton interpolation must agree, and both
    must equal the oracle."""
    from paper_1103_4697_gb300.native import OPT_INTERP_GEMM, OPT_POINTS

    ctx.set_option(OPT_POINTS, 1)          # integer points: the routes under test
    fs, gs = [], []
    for i in range(37):
        bits = 8 if i % 2 else 40
        f, g = W.small_dense_pair(700 + i, 6, bits)
        fs.append(f)
        gs.append(g)
    got = ctx.resultant_batch(fs, gs)
    ctx.set_option(OPT_INTERP_GEMM, 0)
    try:
        newton = ctx.resultant_batch(fs, gs)
    finally:
        ctx.set_option(OPT_INTERP_GEMM, 1)
        ctx.set_option(OPT_POINTS, 0)
    assert got == newton
    for f, g, r in zip(fs, gs, got):
        assert r == list(O.res_bareiss(f, g))


def test_tensor_core_contraction_matches_integer_pipes(ctx):
    """The interpolation contractions of up to 256 points run on the tensor cores
    (bf16 digits, exact fp32 sums); larger ones on the integer pipes.  Point counts
    odd and even (a symmetric set one point larger), 150 pairs sharing one count
    (two pair tiles), and a count above the tensor-core limit in the same batch:
    the results equal those of the integer-pipe contraction and the oracle."""
    from paper_1103_4697_gb300.native import OPT_INTERP_TC, OPT_POINTS

    ctx.set_option(OPT_POINTS, 1)          # integer points: the routes under test
    fs, gs = [], []
    for i in range(150):                              # P = 17: two tiles of 128 pairs
        f, g = W.small_dense_pair(900 + i, 4, 12)
        fs.append(f)
        gs.append(g)
    for d, bits in ((3, 30), (7, 20), (10, 16), (15, 8), (16, 8), (23, 6)):   # P = 10, 50, 101, 226, 257, 530
        f, g = W.small_dense_pair(950 + d, d, bits)
        fs.append(f)
        gs.append(g)
    got = ctx.resultant_batch(fs, gs)
    ctx.set_option(OPT_INTERP_TC, 0)
    try:
        ref = ctx.resultant_batch(fs, gs)
    finally:
        ctx.set_option(OPT_INTERP_TC, 1)
        ctx.set_option(OPT_POINTS, 0)
    assert got == ref
    for q in (0, 77, 149, 150, 151):
        assert got[q] == list(O.res_bareiss(fs[q], gs[q]))
    rng = random.Random(11)
    for q in range(152, len(fs)):
        for a in (rng.randint(-10 ** 6, 10 ** 6), rng.randint(-10 ** 6, 10 ** 6)):
            assert _poly_eval(got[q], a) == O.res_at_prs(fs[q], gs[q], a)


def test_pipelined_batch_matches_one_piece(ctx):
    """A one-shot batch of 2048 pairs or more runs in chunks of 1024 on two internal
    streams (copies and host work overlap the kernels); the results equal those of
    the same batch run in one piece, for resultants and for res(f, f_y)."""
    from paper_1103_4697_gb300.native import OPT_PIPELINE

    fs, gs = [], []
    for i in range(2600):
        f, g = W.small_dense_pair(3000 + i, 3 + i % 3, 10 + i % 7)
        fs.append(f)
        gs.append(g)
    got = ctx.resultant_batch(fs, gs)
    got_d = ctx.discriminant_res_batch(fs)
    ctx.set_option(OPT_PIPELINE, 0)
    try:
        ref = ctx.resultant_batch(fs, gs)
        ref_d = ctx.discriminant_res_batch(fs)
    finally:
        ctx.set_option(OPT_PIPELINE, 1)
    assert got == ref and got_d == ref_d
    for q in (0, 1023, 1024, 2047, 2048, 2599):
        assert got[q] == list(O.res_subres(fs[q], gs[q]))
    assert got_d[2599] == list(O.disc_res(fs[2599]))


def _bimul(a, b):
    """Product of two bivariate polynomials given as rows (row j = x-coefficients of y^j)."""
    nx = len(a[0]) + len(b[0]) - 1
    out = [[0] * nx for _ in range(len(a) + len(b) - 1)]
    for i, ra in enumerate(a):
        for j, rb in enumerate(b):
            for u, ca in enumerate(ra):
                for v, cb in enumerate(rb):
                    out[i + j][u + v] += ca * cb
    return out


def test_register_form_matches_shared_memory_form(ctx):
    """Pairs of shape (N, N), (N, N-1), (N-1, N) for every N of the register form
    (2..32) are solved with the polynomials in registers; pairs even in y (the
    remainder sequence is not normal at any point), pairs whose leading coefficient
    vanishes at integer points, pairs with a planted common factor and a shape
    outside the register form ride along.  With the register form off every
    subproblem runs on shared memory: both must agree with each other and with the
    oracle, and the register run must have sent warps to the shared-memory redo."""
    from paper_1103_4697_gb300.native import OPT_REGISTER_FORM, OPT_STATS

    rng = random.Random(23)

    def rnd(ny, nx, even=False):
        rows = [[rng.randint(-40, 40) for _ in range(nx + 1)] for _ in range(ny + 1)]
        if even:
            rows = [r if j % 2 == 0 else [0] * (nx + 1) for j, r in enumerate(rows)]
        if not any(rows[-1]):
            rows[-1][0] = 1
        return rows

    fs, gs = [], []
    for N in range(2, 33):
        for m, n in ((N, N), (N, N - 1), (N - 1, N)):
            fs.append(rnd(m, 1))
            gs.append(rnd(n, 1))
    for N in (4, 6, 10, 20):
        fs.append(rnd(N, 1, even=True))
        gs.append(rnd(N, 1, even=True))
    for N in (5, 12, 20):
        h = rnd(2, 1)
        fs.append(_bimul(h, rnd(N - 2, 1)))
        gs.append(_bimul(h, rnd(N - 2, 1)))
    for N in (3, 9, 16):
        f, g = rnd(N, 1), rnd(N, 1)
        f[-1] = [-3, 1]        # lc_y f = x - 3 vanishes at x = 3 for every prime
        fs.append(f)
        gs.append(g)
    fs.append(rnd(7, 2))
    gs.append(rnd(3, 2))
    ctx.set_option(OPT_STATS, 1)
    try:
        got = ctx.resultant_batch(fs, gs)
        st = ctx.stats()
        ctx.set_option(OPT_REGISTER_FORM, 0)
        shared = ctx.resultant_batch(fs, gs)
        st0 = ctx.stats()
    finally:
        ctx.set_option(OPT_REGISTER_FORM, 1)
        ctx.set_option(OPT_STATS, 0)
    assert got == shared
    assert st["redo_warps"] > 0 and st0["redo_warps"] == 0
    prng = random.Random(5)
    for f, g, r in zip(fs, gs, got):
        if max(len(f), len(g)) <= 11:
            assert r == _oracle(f, g)
        else:
            for a in (prng.randint(-10 ** 6, 10 ** 6), prng.randint(-10 ** 6, 10 ** 6)):
                assert _poly_eval(r, a) == O.res_at_prs(f, g, a)
    planted = got[3 * 31 + 4: 3 * 31 + 7]
    assert all(r == [] or all(c == 0 for c in r) for r in planted)


def test_drop_unlucky_matches_formal_degrees(ctx):
    """Dropping unlucky points (a leading coefficient vanishes there) for spare
    points, and unlucky primes (a leading coefficient vanishes identically) for the
    next table primes, gives the same resultants as keeping them with formal
    degrees; the counters show that points and primes were actually dropped."""
    from paper_1103_4697_gb300.api import primes
    from paper_1103_4697_gb300.native import OPT_DROP_UNLUCKY

    p0, p1 = primes(2)
    pt_f = [[1, 2, -1], [0, 1], [0, -6, 1, 1]]                 # lc vanishes at x = 0, 2 (and -3)
    pt_g = [[2, -1], [1, 0, 1], [-2, 1]]                       # lc vanishes at x = 2
    pr_f = [[3, 1, 4], [1, 5], [p0 * p1, 0, p0 * p1 * 7]]      # lc = 0 mod p0 and mod p1
    pr_g = [[2, 7], [1, 8, 2], [9]]
    rng = random.Random(17)
    fs = [pt_f, pr_f] + [[[rng.randint(-9, 9) for _ in range(4)] for _ in range(rng.randint(1, 6))] for _ in range(30)]
    gs = [pt_g, pr_g] + [[[rng.randint(-9, 9) for _ in range(3)] for _ in range(rng.randint(1, 6))] for _ in range(30)]
    formal = ctx.resultant_batch(fs, gs)
    ctx.set_option(OPT_DROP_UNLUCKY, 1)
    try:
        dropped = ctx.resultant_batch(fs, gs)
        st = ctx.stats()
        d1 = ctx.discriminant_res(pt_f)
    finally:
        ctx.set_option(OPT_DROP_UNLUCKY, 0)
    assert dropped == formal
    assert st["dropped_points"] >= 2 and st["dropped_primes"] >= 2
    for f, g, r in zip(fs, gs, formal):
        assert r == _oracle(f, g)
    assert d1 == ctx.discriminant_res(pt_f) == list(O.disc_res(pt_f))


def test_graph_replay_and_autotuned_blocks(ctx):
    """A resident batch run twice replays its captured CUDA graph the second time;
    results are identical with graphs off, and the autotuner has picked a block
    size for the batch's degree bucket."""
    from paper_1103_4697_gb300.native import OPT_GRAPH, OPT_STATS

    F, G = W.deg20_batch_arrays(96, 9000, d=7, bits=12)
    ctx.set_option(OPT_STATS, 1)
    res = ctx.upload_pairs(F, G)
    res.run()                      # first sighting of the plan: plain launches
    first = res.fetch()
    res.run()                      # second: captured, then launched as a graph
    res.run()                      # third: replayed
    st = ctx.stats()
    second = res.fetch()
    ctx.set_option(OPT_GRAPH, 0)
    try:
        res.run()
        plain = res.fetch()
        st_plain = ctx.stats()
    finally:
        ctx.set_option(OPT_GRAPH, 1)
        ctx.set_option(OPT_STATS, 0)
    res.free()
    assert st["graph_replayed"] == 1 and st_plain["graph_replayed"] == 0
    assert first == second == plain
    for q in (0, 37, 95):
        assert first[q] == list(O.res_subres(F[q], G[q]))


def test_step_graph_replay(ctx):
    """From the fourth run of a resident batch the whole step (bounds, plan check,
    stages) is one graph launch with no host planning in between; its results equal
    those of the planned runs and the oracle.  Changing an option that shapes the plan
    (extra primes) goes back to planning; an interleaved other batch that evicts
    nothing leaves the step graph valid."""
    from paper_1103_4697_gb300.native import OPT_EXTRA_PRIMES, OPT_STATS

    F, G = W.deg20_batch_arrays(160, 7000, d=9, bits=14)
    ctx.set_option(OPT_STATS, 1)
    res = ctx.upload_pairs(F, G)
    outs, modes, kernels = [], [], []
    for _ in range(5):
        res.run()
        st = ctx.stats()
        outs.append(res.fetch())
        modes.append(st["graph_replayed"])
        kernels.append(st["kernels"])
    assert modes == [0, 1, 1, 2, 2], modes
    # every run launches the two bounds kernels; the step graph adds the plan check
    assert kernels[3] == kernels[2] + 1
    assert all(o == outs[0] for o in outs)
    other = ctx.upload_pairs(*W.deg20_batch_arrays(8, 7500, d=5, bits=10))
    other.run()
    other.free()
    res.run()
    assert ctx.stats()["graph_replayed"] == 2 and res.fetch() == outs[0]
    ctx.set_option(OPT_EXTRA_PRIMES, 1)
    try:
        res.run()
        assert ctx.stats()["graph_replayed"] == 0 and res.fetch() == outs[0]
    finally:
        ctx.set_option(OPT_EXTRA_PRIMES, 0)
        ctx.set_option(OPT_STATS, 0)
    res.free()
    rng = random.Random(4)
    for q in rng.sample(range(160), 4):
        assert outs[0][q] == list(O.res_subres(F[q], G[q]))


def test_one_shot_calls_reuse_their_graphs():
    """gbr_resultant_batch called again with inputs of the same shape keeps its batch,
    plan and graphs: from the fifth call the whole step is one graph.  New contents in
    the same buffers whose plan still fits (each row reversed: same degrees and bounds)
    run from that graph and give their own, correct results; contents that need more
    primes make the device check decline the graph, and the call plans again."""
    from paper_1103_4697_gb300.api import Context
    from paper_1103_4697_gb300.native import OPT_STATS

    F, G = W.deg20_batch_arrays(200, 8100, d=8, bits=12)
    F[:, :, 0][F[:, :, 0] == 0] = 1          # reversed rows keep their degrees
    with Context(device=0, mem_budget=2 << 30) as c:
        c.set_option(OPT_STATS, 1)
        modes, outs = [], []
        for _ in range(6):
            outs.append(c.resultant_batch(F, G))
            modes.append(c.stats()["graph_replayed"])
        assert modes == [0, 0, 1, 1, 2, 2], modes
        assert all(o == outs[0] for o in outs)
        rng = random.Random(6)
        for q in rng.sample(range(200), 3):
            assert outs[0][q] == list(O.res_subres(F[q], G[q]))
        for j in range(9):                                  # reverse row j (x-degree 8 - j) in place
            F[:, j, :9 - j] = F[:, j, 8 - j::-1].copy()
        got = c.resultant_batch(F, G)
        assert c.stats()["graph_replayed"] == 2
        for q in rng.sample(range(200), 6):
            a = rng.randint(-2 ** 31, 2 ** 31)
            assert _poly_eval(got[q], a) == O.res_at_prs(F[q], G[q], a), q
        F[7] <<= 30                                          # pair 7 now needs more primes
        got2 = c.resultant_batch(F, G)
        assert c.stats()["graph_replayed"] == 0
        assert got2[7] == list(O.res_subres(F[7], G[7]))
        assert got2[:7] == got[:7] and got2[8:] == got[8:]


def test_device_bound_is_rigorous_and_tight(ctx):
    """The device evaluates the scaled Hadamard bound in single precision with
    upward rounding and error margins; it must never fall below the host's
    double-precision value of the same bound (that would leave too few primes) and
    stays within a small margin above it."""
    from paper_1103_4697_gb300.api import resultant_info

    ps = W.mixed_batch(3, 96)
    d20 = W.deg20_batch(8)
    fc, gc = W.conic_curves(4)
    cases = [(f, g, 0) for f, g in zip(ps.f, ps.g)] + [(f, g, 0) for f, g in zip(d20.f, d20.g)]
    cases += [(fc, gc, 0), (fc, None, 1), (d20.f[0], None, 1)]
    for var in (1, 0):
        res = ctx.upload_pairs([c[0] for c in cases[:-2]], [c[1] for c in cases[:-2]], var=var)
        disc = ctx.upload_pairs([c[0] for c in cases[-2:]], var=var, disc=True)
        try:
            res.run()
            disc.run()
            dev = res.plan() + disc.plan()
        finally:
            res.free()
            disc.free()
        for (f, g, dflag), d in zip(cases, dev):
            h = resultant_info(f, g, var=var, disc=bool(dflag))
            assert (d["m"], d["n"]) == (h["m"], h["n"])
            if h["deg_bound"] < 0:
                assert d["primes"] == 0
                continue
            assert d["log2_bound"] >= h["log2_bound"] - 1e-9 * max(1.0, abs(h["log2_bound"]))
            assert d["log2_bound"] <= h["log2_bound"] + 0.01 + 0.002 * (h["m"] + h["n"])
            assert h["primes"] <= d["primes"] <= h["primes"] + 1
