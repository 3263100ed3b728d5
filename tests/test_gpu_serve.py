"""Serving (continuous batching): each result is the same alone and in the mix."""

import random
import time

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


def test_mixed_stream_matches_alone_and_oracle(ctx):
    from paper_1103_4697_gb300.native import JOB_DISC, JOB_GCD, JOB_RESULTANT

    reqs = W.serving_stream(5, 240, rate=1e9, dlo=3, dhi=9, blo=8, bhi=64)
    tickets = []
    for k, r in enumerate(reqs):
        if r.kind == "res":
            kind = JOB_DISC if k % 7 == 0 else JOB_RESULTANT
            tickets.append((ctx.submit(kind, r.a, r.b), kind, r))
        else:
            tickets.append((ctx.submit(JOB_GCD, r.a, r.b), JOB_GCD, r))
        if k % 40 == 0:
            time.sleep(0.002)          # let some batches start while others arrive
    results = [ctx.poll(t, -1) for t, _, _ in tickets]
    rng = random.Random(1)
    for (t, kind, r), got in zip(tickets, results):
        if kind == JOB_GCD:
            assert got == list(O.gcd_z(r.a, r.b))
        elif kind == JOB_DISC:
            assert got == list(O.disc_res(r.a))
        else:
            if r.planted:
                assert got == []
            assert got == list(O.res_subres(r.a, r.b))
    # the same jobs alone, one call each, give identical results
    for (t, kind, r), got in rng.sample(list(zip(tickets, results)), 20):
        if kind == JOB_GCD:
            assert ctx.gcd(r.a, r.b) == got
        elif kind == JOB_DISC:
            assert ctx.discriminant_res(r.a) == got
        else:
            assert ctx.resultant(r.a, r.b) == got
    st = ctx.serve_stats()
    assert st["completed"] == st["submitted"] == len(reqs)
    assert st["batches"] >= 1


def test_poll_unknown_ticket(ctx):
    from paper_1103_4697_gb300.native import GbrError, ENOTFOUND

    with pytest.raises(GbrError) as e:
        ctx.poll(10 ** 12, 0)
    assert e.value.status == ENOTFOUND


def test_admission_refuses_oversized_job():
    """A job that can never fit the budget fails with ENOMEM; jobs that fit still run."""
    from paper_1103_4697_gb300.api import Context
    from paper_1103_4697_gb300.native import GbrError, ENOMEM, JOB_RESULTANT

    with Context(device=0, mem_budget=4 << 20) as c:
        f, g = W.small_dense_pair(8, 40, 64)     # needs several MiB of residues
        big = c.submit(JOB_RESULTANT, f, g)
        fs, gs = W.small_dense_pair(3, 4, 8)
        small = c.submit(JOB_RESULTANT, fs, gs)
        assert c.poll(small, -1) == list(O.res_subres(fs, gs))
        with pytest.raises(GbrError) as e:
            c.poll(big, -1)
        assert e.value.status == ENOMEM


def test_full_mix_burst_every_request(ctx):
    """Full request mix (degree 5..30, 8..64-bit): a burst of 1200 requests overlaps on
    the workers' streams; every gcd is checked exactly and every resultant at two
    random 32-bit points (planted pairs must give 0)."""
    import oracle_tasks as T
    from paper_1103_4697_gb300.native import JOB_GCD, JOB_RESULTANT

    reqs = W.serving_stream(55, 1200, rate=1e12)
    tickets = [ctx.submit(JOB_RESULTANT if r.kind == "res" else JOB_GCD, r.a, r.b) for r in reqs]
    out = [ctx.poll(t, -1) for t in tickets]
    rng = random.Random(2)
    gi = [i for i, r in enumerate(reqs) if r.kind == "gcd"]
    ri = [i for i, r in enumerate(reqs) if r.kind != "gcd"]
    pts = {i: [rng.randint(-2 ** 31, 2 ** 31) for _ in range(2)] for i in ri}
    with T.pool() as pool:
        gw = pool.map(T.gcd_exact, [(reqs[i].a, reqs[i].b) for i in gi], chunksize=8)
        rw = pool.map(T.res_points, [(reqs[i].a, reqs[i].b, pts[i]) for i in ri], chunksize=8)
    for i, w in zip(gi, gw):
        assert out[i] == w, i
    for i, w in zip(ri, rw):
        got = []
        for a in pts[i]:
            v = 0
            for c in reversed(out[i]):
                v = v * a + c
            got.append(v)
        assert got == w, i
        if reqs[i].planted:
            assert out[i] == [], i


def test_wait_any_returns_every_job_once(ctx):
    """gbr_wait_any hands out finished jobs in completion order: every ticket once,
    with the result gbr_poll would give, mixed with tickets consumed by polls."""
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300.native import JOB_GCD, JOB_RESULTANT

    reqs = W.serving_stream(9, 120, rate=1e9, dlo=3, dhi=8, blo=8, bhi=40)
    t0 = N.lib().gbr_clock()
    tickets = {}
    for r in reqs:
        kind = JOB_RESULTANT if r.kind == "res" else JOB_GCD
        tickets[ctx.submit(kind, r.a, r.b)] = (kind, r)
    # a few tickets are taken by polls first; wait_any must skip them
    polled = {}
    for t in list(tickets)[:5]:
        polled[t] = ctx.poll(t, -1)
    got, times = {}, []
    while True:
        x = ctx.wait_any(2000)
        if x is None:
            break
        t, res, td = x
        assert t in tickets and t not in got and t not in polled
        got[t] = res
        times.append(td)
    assert len(got) + len(polled) == len(tickets)
    assert times == sorted(times) and times[0] >= t0
    for t, res in list(got.items())[:40] + list(polled.items()):
        kind, r = tickets[t]
        if kind == JOB_GCD:
            assert res == list(O.gcd_z(r.a, r.b))
        else:
            assert res == list(O.res_subres(r.a, r.b))
    assert ctx.wait_any(0) is None                 # nothing outstanding
