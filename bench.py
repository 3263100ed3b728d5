#!/usr/bin/env python3
"""Benchmark: bit-exact res_y(f, g) solves per second on the batched degree-20
workload (4096 dense pairs of total degree 20, 16-bit signed coefficients,
pair i drawn from seed 2000 + i), one device-resident batch per step; plus
serving p50/p99 latency on a Poisson stream of mixed resultant/gcd requests.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs its own batch of
4096 pairs (seeds offset by rank, weak scaling, no collective on the data
path); the barrier and the max-over-ranks timing use torch.distributed.
"""

from __future__ import annotations

import argparse
import ctypes as C
import functools
import hashlib
import json
import math
import multiprocessing as mp
import os
import random
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "bit-exact res_y(f,g) solves/sec (deg 20; batched 4096 pairs); serving p50/p99"
PAIRS, DEG, BITS, BASE_SEED = 4096, 20, 16, 2000


# --------------------------------------------------------------------------- distributed helpers


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_seed_base(rank: int, pairs: int = PAIRS) -> int:
    """Rank r solves pairs with seeds BASE_SEED + r * pairs + i (rank 0: the headline seeds)."""
    return BASE_SEED + rank * pairs


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples during the timed region (every 200 ms)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- CPU oracle baseline


def _oracle_pair(seed: int):
    import oracle as O
    from paper_1103_4697_gb300 import workloads as W

    f, g = W.small_dense_pair(seed, DEG, BITS)
    t = time.perf_counter()
    r = O.res_evalz(f, g)
    return time.perf_counter() - t, len(r)


def oracle_baseline(pairs_per_core: int = 1, cores: int | None = None) -> dict:
    """The oracle as it stands (exact evaluation/interpolation over Z, res_evalz) on a
    bounded sample of the workload's pairs, one pair per process on every host core."""
    cores = cores or os.cpu_count() or 1
    n = max(1, cores * pairs_per_core)
    seeds = [BASE_SEED + i for i in range(n)]
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_pair, seeds, chunksize=1)
    wall = time.perf_counter() - t
    return {"value": n / wall, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} of the {PAIRS} pairs (seeds {BASE_SEED}..{BASE_SEED + n - 1}), res_evalz, "
                      f"{wall:.1f} s wall, mean {statistics.mean(r[0] for r in res):.1f} s per pair"}


# --------------------------------------------------------------------------- serving


def _serve_prepare(reqs):
    """Requests -> packed job descriptors (and the buffers they point into)."""
    from paper_1103_4697_gb300 import api
    from paper_1103_4697_gb300 import native as N

    keep = api._Packed()
    jobs = []
    for r in reqs:
        kind = N.JOB_RESULTANT if r.kind == "res" else N.JOB_GCD
        jobs.append(api._job(kind, r.a, r.b, 1, keep))
    return jobs, keep


def _serve_run(ctx, jobs, arrivals):
    """A submitter thread releases each job at its arrival time; this thread takes
    finished jobs with gbr_wait_any (blocking in the library, without the GIL) and
    keeps the library's completion time of each, on perf_counter's clock."""
    from paper_1103_4697_gb300 import native as N

    L = N.lib()
    n = len(jobs)
    done = [0.0] * n
    index = {}
    # both clocks are CLOCK_MONOTONIC on Linux; the offset removes any difference
    off = time.perf_counter() - L.gbr_clock()
    t0 = time.perf_counter() + 0.01

    def submitter():
        for i, j in enumerate(jobs):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            t = C.c_uint64()
            N.check(L.gbr_submit(ctx.handle, C.byref(j), C.byref(t)), ctx.handle)
            index[t.value] = i

    th = threading.Thread(target=submitter)
    th.start()
    out = N.BigPoly()
    tk = C.c_uint64()
    td = C.c_double()
    left = n
    while left:
        st = L.gbr_wait_any(ctx.handle, 100, C.byref(tk), C.byref(out), C.byref(td))
        if st in (N.ETIMEOUT, N.EAGAIN, N.ENOTFOUND):
            if st == N.ENOTFOUND:
                time.sleep(1e-4)                    # nothing submitted yet
            continue
        assert st == N.OK, f"serving request failed with status {st}"
        while tk.value not in index:                # the submitter records the ticket
            time.sleep(1e-6)
        done[index[tk.value]] = td.value + off
        L.gbr_free_result(ctx.handle, C.byref(out))
        left -= 1
    th.join()
    return t0, done


def _latency(t0, done, arrivals, rate):
    lat = sorted((done[i] - (t0 + arrivals[i])) * 1e3 for i in range(len(done)))
    span = max(done) - t0
    return {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[int(len(lat) * 0.99)], "throughput_rps": len(done) / span,
            "offered_rps": rate, "requests": len(done)}


def serving_run(ctx, n_burst: int = 1500, n_stream: int = 6000, load: float = 0.8, seed: int = 5,
                capacity: float | None = None) -> dict:
    """Open-loop Poisson stream of mixed resultant/gcd requests (degree log-uniform
    5..30, 8..64-bit coefficients, 10 % planted factors): capacity from a burst, then
    a stream at `load` x capacity; latency = completion - scheduled arrival."""
    from paper_1103_4697_gb300 import workloads as W

    if capacity is None:
        burst = W.serving_stream(seed, n_burst, rate=1e12)
        jb, kb = _serve_prepare(burst)
        _serve_run(ctx, jb, [0.0] * len(jb))                   # warm-up: caches, tables, streams
        t0, done = _serve_run(ctx, jb, [0.0] * len(jb))
        capacity = len(jb) / (max(done) - t0)
    rate = load * capacity
    stream = W.serving_stream(seed + 1, n_stream, rate=rate)
    js, ks = _serve_prepare(stream)
    arrivals = [r.t_arrive for r in stream]
    t0, done = _serve_run(ctx, js, arrivals)
    out = _latency(t0, done, arrivals, rate)
    out.update({"capacity_rps": capacity,
                "mix": "50/50 res_y/gcd, degree log-uniform 5..30, 8..64-bit, 10% planted",
                "stats": ctx.serve_stats()})
    return out


def serving_loads(ctx, n: int = 100_000, seed: int = 5, n_burst: int = 3000, n_single: int = 1000) -> dict:
    """The serving configuration at its stated size: one Poisson stream of n mixed
    requests (drawn once at unit rate; a load scales its arrival times), replayed at 0.5,
    0.8 and 0.95 of the capacity measured on a burst; and the same mix run one request
    per synchronous call (gbr_resultant / gbr_gcd) as the like-for-like baseline."""
    from paper_1103_4697_gb300 import api
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300 import workloads as W

    L = N.lib()
    burst = W.serving_stream(seed, n_burst, rate=1e12)
    jb, kb = _serve_prepare(burst)
    _serve_run(ctx, jb, [0.0] * len(jb))
    t0, done = _serve_run(ctx, jb, [0.0] * len(jb))
    capacity = len(jb) / (max(done) - t0)
    t = time.perf_counter()
    stream = W.serving_stream(seed + 1, n, rate=1.0)
    js, ks = _serve_prepare(stream)
    prep_s = time.perf_counter() - t
    # untimed warm-up over the stream itself as a burst: tables, point sets and tuned
    # block sizes for every shape it holds
    _serve_run(ctx, js[:20000], [0.0] * min(20000, len(js)))
    loads = {}
    for load in (0.5, 0.8, 0.95):
        rate = load * capacity
        arrivals = [r.t_arrive / rate for r in stream]
        t0, done = _serve_run(ctx, js, arrivals)
        loads[str(load)] = _latency(t0, done, arrivals, rate)
    # one request per call, the same mix
    single = stream[:n_single]
    keep = api._Packed()
    t = time.perf_counter()
    for r in single:
        o = N.BigPoly()
        if r.kind == "res":
            df, dg = api.pack_bipolys([r.a], keep), api.pack_bipolys([r.b], keep)
            N.check(L.gbr_resultant(ctx.handle, C.cast(api._ptr(df), C.POINTER(N.BiPoly)),
                                    C.cast(api._ptr(dg), C.POINTER(N.BiPoly)), 1, C.byref(o)), ctx.handle)
        else:
            dp, dq = api.pack_upolys([r.a], keep), api.pack_upolys([r.b], keep)
            N.check(L.gbr_gcd(ctx.handle, C.cast(api._ptr(dp), C.POINTER(N.UPoly)),
                              C.cast(api._ptr(dq), C.POINTER(N.UPoly)), C.byref(o)), ctx.handle)
        L.gbr_free_result(ctx.handle, C.byref(o))
    one_rps = n_single / (time.perf_counter() - t)
    return {"capacity_rps": capacity, "loads": loads, "requests_per_load": n,
            "one_request_per_call_rps": one_rps, "one_request_per_call_sample": n_single,
            "host_prepare_s": prep_s, "stats": ctx.serve_stats(),
            "mix": "50/50 res_y/gcd, degree log-uniform 5..30, 8..64-bit, 10% planted (seed 6)"}


# --------------------------------------------------------------------------- roofline counts


def _pow_cost(e: int) -> int:
    """Montgomery products of the kernels' square-and-multiply power x^e (e >= 1)."""
    return bin(e).count("1") + e.bit_length() - 1


@functools.lru_cache(maxsize=None)
def regform_ops(m: int, n: int, tf: int, tg: int, p: int, seg: int = 512, radix: int = 2) -> dict:
    """Operations the register-form kernel executes for one (prime, point) subproblem of
    a pair of y-degrees (m, n) in one of its shapes (N, N), (N, N-1), (N-1, N), counted
    from its code: the evaluation's Horner steps in Shoup form ((tf + tg) / radix per
    point, tf and tg the numbers of stored coefficients, rows of x-degree e counting
    e + 1; radix 2: even and odd parts for +-a, radix 4: the four parts in x^4 for the
    quartic set's +-a, +-i a) and the combine (radix 2: E + a O, one product per row and
    point pair; radix 4: a^t P_t and i (A_1 - A_3), four products per row and point
    quadruple, plus a^3, a^4 per point); elimination: for (N, N) the
    first multiply-subtract row and alpha^N, then N - 1 normal rounds (round of degree d:
    one fused two-product and d - 1 fused three-product updates, and the scalars z^2,
    z alpha, q0, Q z^2 and, after the first round, the telescoped divisor), the two
    final products of numerator and denominator; then the batch inversion that forms
    the quotient (four products per value, and per segment of `seg` values the scans
    and one Fermat inverse x^(p-2))."""
    N = max(m, n)
    mul = (m + n + 2) / 2 + 2 + 4 + (12 + _pow_cost(p - 2)) / seg
    if radix == 4:
        mul += (m + n + 2) / 2 + 4
    mulsub, fma2, fma3 = 0, 0, 0
    if m == n:
        mulsub += N
        mul += _pow_cost(N)
    for d in range(N - 1, 0, -1):
        mul += 3 + (0 if d == N - 1 else 1)
        mulsub += 1
        fma2 += 1
        fma3 += d - 1
    return {"shoup": (tf + tg) / radix, "mul": mul, "mulsub": mulsub + fma2, "fma3": fma3}


def evalres_roofline(F, G, plans: list[dict], table: list[int], cal: dict, quartic: bool = False) -> dict:
    """Modular products the evaluation + elimination stage executes for a batch of
    dense pairs (pair q on the first plans[q]["primes"] primes of the table, at the
    points of its set: the symmetric integers 0, +-1, ... covering deg_bound + 1, or with
    `quartic` the set 0, +-a, +-i a, a = 1..ceil(deg_bound / 4), in radix 4), and the time
    they would take if every operation ran at its calibrated rate on this GPU."""
    import numpy as np

    ops = {"shoup": 0.0, "mul": 0.0, "mulsub": 0.0, "fma3": 0.0}
    textbook = 0

    def shape(A):
        """(y-degree, stored coefficients) of rows A[j][i] (an array or ragged lists)."""
        rows = [np.nonzero(np.asarray(r, dtype=object) != 0)[0] for r in A]
        deg_y = max((j for j, xs in enumerate(rows) if len(xs)), default=-1)
        return deg_y, sum((int(rows[r][-1]) + 1) if len(rows[r]) else 1 for r in range(deg_y + 1))

    for q in range(len(F)):
        if plans[q]["primes"] <= 0:
            continue
        D = plans[q]["deg_bound"]
        points = 4 * ((D + 3) // 4) + 1 if quartic else 2 * ((D + 1) // 2) + 1
        primes = table[:plans[q]["primes"]]
        shapes = [shape(F[q]), shape(G[q])]
        (m, tf), (n, tg) = shapes
        textbook += len(primes) * (D + 1) * (tf + tg + 2 * m * n)
        for p in primes:
            for k, v in regform_ops(m, n, tf, tg, p, min(points, 512), 4 if quartic else 2).items():
                ops[k] += v * points
    products = ops["shoup"] + ops["mul"] + 2 * ops["mulsub"] + 3 * ops["fma3"]
    ideal_s = (ops["shoup"] / cal["shoup_per_s"] + ops["mul"] / cal["modmul_per_s"]
               + ops["mulsub"] / cal["mulsub_per_s"] + ops["fma3"] / cal["fma3_per_s"])
    return {"products": products, "textbook_products": textbook, "ideal_s": ideal_s,
            "ops": {k: v for k, v in ops.items()}}


# --------------------------------------------------------------------------- the five configurations


def _oracle_job(job):
    """One oracle computation for the per-configuration CPU figures: (name, seconds)."""
    import oracle as O
    from paper_1103_4697_gb300 import workloads as W

    kind, arg = job
    t = time.perf_counter()
    if kind == "c1_res":
        f, g = W.small_dense_pair(1)
        O.res_bareiss(f, g)
    elif kind == "c1_gcd":
        f, g = W.small_dense_pair(1)
        O.gcd_z(list(f[0]), list(g[0]))
    elif kind == "c2_res":
        f, g = W.deg20_pair(2)
        O.res_evalz(f, g)
    elif kind == "c2_disc":
        f, g = W.deg20_pair(2)
        O.disc_res(f, "evalz")
    elif kind == "c3_res":
        ps = W.mixed_batch(3, arg + 1)
        O.res_evalz(ps.f[arg], ps.g[arg])
    elif kind == "c3_gcd":
        P, Q, _ = W.gcd_batch(3, arg + 1)
        O.gcd_z(P[arg], Q[arg])
    elif kind == "c4_res":
        f, g = W.conic_curves(4)
        O.res_evalz(f, g)
    elif kind == "c5":
        reqs = W.serving_stream(5, arg + 1, rate=1.0)
        r = reqs[arg]
        (O.res_subres if r.kind == "res" else O.gcd_z)(r.a, r.b)
    return kind, time.perf_counter() - t


def _stage_roofline(ctx, st: dict, fs, gs, plans, cal: dict) -> dict:
    """Stage times of the last run and the evaluation stage against its own operation mix
    at the calibrated rates (register-form count; small runs are launch bound)."""
    from paper_1103_4697_gb300 import api

    rl = evalres_roofline(fs, gs, plans, api.primes(max(p["primes"] for p in plans) or 1), cal,
                          st.get("quad_pairs", 0) * 2 > len(fs))
    ms = st["evalres_ms"]
    achieved = rl["products"] / (ms * 1e-3) if ms > 0 else 0.0
    return {"stages_ms": {k: st[k] for k in ("bounds_ms", "reduce_ms", "evalres_ms", "interp_ms", "crt_ms")},
            "note": "bounds_ms runs from the bounds kernels to the first stage kernel: for a call that is not "
                    "replayed from a step graph it includes the host plan and its upload",
            "evalres": {"bound": "alu", "products": rl["products"], "achieved_Tmodmul_s": achieved / 1e12,
                        "peak_Tmodmul_s": rl["products"] / rl["ideal_s"] / 1e12 if rl["ideal_s"] else None,
                        "frac": achieved * rl["ideal_s"] / rl["products"] if rl["products"] else None}}


def configs_block(ctx, cal: dict, serve_requests: int = 100_000) -> dict:
    """Every configuration measured on this GPU beside the plain one-pair-per-launch GPU
    path and the oracle on the host cores (a bounded sample each, timed in a spawn pool
    before any GPU work of this block):
      1  one dense degree-6 pair: res_y(f, g) and gcd(f(x, 0), g(x, 0)), one call each;
      2  one dense degree-20 pair: res_y(f, g) and res_y(f, f_y), one call each;
      3  4096 mixed pairs (degrees 4..16, 8..32-bit, 25 % planted) as one resident batch
         and 4096 gcds (degrees 30..200) through the C ABI, with their one-per-call rates;
      4  the conic product against a dense degree-24 curve: res_y(f, g), res_y(f, f_y);
      5  a Poisson stream of mixed requests at 0.5, 0.8 and 0.95 of the measured
         capacity (p50/p99 latency, throughput), and the same mix one request per call."""
    import torch

    import oracle as O
    from paper_1103_4697_gb300 import api
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300 import workloads as W

    L = N.lib()
    cores = os.cpu_count() or 1
    jobs = [("c1_res", 0), ("c1_gcd", 0), ("c2_res", 0), ("c2_disc", 0), ("c4_res", 0)]
    jobs += [("c3_res", i) for i in range(8)] + [("c3_gcd", i) for i in range(8)] + [("c5", i) for i in range(16)]
    # a bounded sample: every job runs on its own core; a job still running at the cap
    # counts with the cap as its time (a lower bound on the oracle's cost)
    cap_s = 30.0
    t0 = time.perf_counter()
    pool = mp.get_context("spawn").Pool(cores)
    pend = [(job, pool.apply_async(_oracle_job, (job,))) for job in jobs]
    per, capped = {}, {}
    for job, r in pend:
        left = cap_s - (time.perf_counter() - t0)
        try:
            k, sec = r.get(timeout=max(left, 0.01))
        except mp.TimeoutError:
            k, sec = job[0], cap_s
            capped[k] = capped.get(k, 0) + 1
        per.setdefault(k, []).append(sec)
    pool.terminate()
    owall = time.perf_counter() - t0

    def oracle_rate(kind):
        v = per[kind]
        out = {"s_per_job_1core": statistics.mean(v), "jobs": len(v)}
        if capped.get(kind):
            out["capped_jobs"] = capped[kind]
            out["note"] = f"{capped[kind]} job(s) still running at the {cap_s:.0f} s cap counted as {cap_s:.0f} s: " \
                          "s_per_job is a lower bound"
        return out

    out = {"oracle_pool": {"cores": cores, "wall_s": owall, "kind": "oracle", "cap_s": cap_s,
                           "sample": "configs 1, 2, 4 whole; 8 pairs and 8 gcds of config 3; 16 requests of config 5"}}
    # 1: one dense degree-6 pair
    f, g = W.small_dense_pair(1)
    p, q = list(f[0]), list(g[0])
    ctx.resultant(f, g)
    ctx.gcd(p, q)
    ctx.set_option(N.OPT_STATS, 1)
    ctx.resultant(f, g)
    rl1 = _stage_roofline(ctx, ctx.stats(), [f], [g], [api.resultant_info(f, g)], cal)
    out["1"] = {"stage_roofline": rl1, "res_ms_per_call": _time_calls(lambda: ctx.resultant(f, g), 20) * 1e3,
                "gcd_ms_per_call": _time_calls(lambda: ctx.gcd(p, q), 20) * 1e3,
                "workload": "one dense pair of total degree 6, coefficients in [-128, 127] (seed 1); "
                            "res_y(f, g) and gcd(f(x, 0), g(x, 0))",
                "oracle_res_ms": per["c1_res"][0] * 1e3, "oracle_gcd_ms": per["c1_gcd"][0] * 1e3,
                "note": "a single pair is the one-pair-per-launch path itself (launch bound)"}
    # 2: one dense degree-20 pair
    f2, g2 = W.deg20_pair(2)
    ctx.resultant(f2, g2)
    ctx.resultant(f2, g2)   # the stage times of a warm call (the first one also builds tables)
    rl2 = _stage_roofline(ctx, ctx.stats(), [f2], [g2], [api.resultant_info(f2, g2)], cal)
    out["2"] = {"stage_roofline": rl2, "res_ms_per_call": _time_calls(lambda: ctx.resultant(f2, g2), 10) * 1e3,
                "disc_ms_per_call": _time_calls(lambda: ctx.discriminant_res(f2), 10) * 1e3,
                "oracle_res_s": per["c2_res"][0], "oracle_disc_s": per["c2_disc"][0],
                "workload": "one dense pair of total degree 20, 16-bit (seed 2); res_y(f, g), res_y(f, f_y)"}
    # 3: the mixed batch, resident, and the gcd batch through the C ABI
    ps = W.mixed_batch(3, PAIRS)
    ctx.set_option(N.OPT_STATS, 1)
    res = ctx.upload_pairs(ps.f, ps.g)
    for _ in range(5):      # from the fourth run on the whole step replays from its graph
        res.run()
    st = ctx.stats()
    rl3 = _stage_roofline(ctx, st, ps.f, ps.g, res.plan(), cal)
    sec = _time_calls(res.run, 10)
    outs = res.fetch()
    assert all(outs[i] == [] for i in range(PAIRS) if ps.planted[i])
    res.free()
    keep = api._Packed()
    df, dg = api.pack_bipolys(ps.f, keep), api.pack_bipolys(ps.g, keep)
    n1 = 64
    t = time.perf_counter()
    for i in range(n1):
        o = N.BigPoly()
        N.check(L.gbr_resultant(ctx.handle, C.cast(api._ptr(df[i:i + 1]), C.POINTER(N.BiPoly)),
                                C.cast(api._ptr(dg[i:i + 1]), C.POINTER(N.BiPoly)), 1, C.byref(o)), ctx.handle)
        L.gbr_free_result(ctx.handle, C.byref(o))
    one_res = n1 / (time.perf_counter() - t)
    P, Q, _H = W.gcd_batch(3, PAIRS)
    dp, dq = api.pack_upolys(P, keep), api.pack_upolys(Q, keep)
    gouts = (N.BigPoly * PAIRS)()
    gtimes = []
    for _ in range(4):
        t = time.perf_counter()
        N.check(L.gbr_gcd_batch(ctx.handle, PAIRS, api._ptr(dp), api._ptr(dq), gouts), ctx.handle)
        gtimes.append(time.perf_counter() - t)
        for i in range(PAIRS):
            L.gbr_free_result(ctx.handle, C.byref(gouts[i]))
    t = time.perf_counter()
    for i in range(n1):
        o = N.BigPoly()
        N.check(L.gbr_gcd(ctx.handle, C.cast(api._ptr(dp[i:i + 1]), C.POINTER(N.UPoly)),
                          C.cast(api._ptr(dq[i:i + 1]), C.POINTER(N.UPoly)), C.byref(o)), ctx.handle)
        L.gbr_free_result(ctx.handle, C.byref(o))
    one_gcd = n1 / (time.perf_counter() - t)
    # both halves as one batch (gbr_mixed_batch) against the two one-shot calls in turn,
    # through the C ABI with packed host buffers; freeing the results is not timed
    rr, rg = (N.BigPoly * PAIRS)(), (N.BigPoly * PAIRS)()

    def free_all():
        for i in range(PAIRS):
            L.gbr_free_result(ctx.handle, C.byref(rr[i]))
            L.gbr_free_result(ctx.handle, C.byref(rg[i]))

    def timed(fn, reps=5):
        ts = []
        for _ in range(reps):
            t = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t)
            free_all()
        return statistics.median(ts[1:])

    mixed_s = timed(lambda: N.check(L.gbr_mixed_batch(ctx.handle, PAIRS, api._ptr(df), api._ptr(dg), 1, rr, PAIRS,
                                                      api._ptr(dp), api._ptr(dq), rg), ctx.handle))
    sep_s = timed(lambda: (N.check(L.gbr_resultant_batch(ctx.handle, PAIRS, api._ptr(df), api._ptr(dg), 1, rr),
                                   ctx.handle),
                           N.check(L.gbr_gcd_batch(ctx.handle, PAIRS, api._ptr(dp), api._ptr(dq), rg), ctx.handle)))
    out["3"] = {"res_solves_per_s": PAIRS / sec, "res_ms_per_batch": sec * 1e3, "stage_roofline": rl3,
                "one_batch_res_plus_gcd_ms": mixed_s * 1e3, "two_calls_res_then_gcd_ms": sep_s * 1e3,
                "one_batch_jobs_per_s": 2 * PAIRS / mixed_s,
                "res_one_pair_per_launch_per_s": one_res,
                "gcd_jobs_per_s": PAIRS / statistics.median(gtimes[1:]),
                "gcd_one_job_per_launch_per_s": one_gcd,
                "oracle_res": oracle_rate("c3_res"), "oracle_gcd": oracle_rate("c3_gcd"),
                "planted_zero": sum(1 for x in ps.planted if x),
                "workload": "4096 pairs, deg_x, deg_y ~ U{4..16}, 8..32-bit, 25% planted (seed 3), one resident "
                            "batch; 4096 gcds of degree 30..200 with a planted degree-5 factor"}
    # 4: the conic product
    f4, g4 = W.conic_curves(4)
    ctx.resultant(f4, g4)
    ctx.resultant(f4, g4)   # the stage times of a warm call (the first one also builds tables)
    rl4 = _stage_roofline(ctx, ctx.stats(), [f4], [g4], [api.resultant_info(f4, g4)], cal)
    out["4"] = {"stage_roofline": rl4, "res_ms_per_call": _time_calls(lambda: ctx.resultant(f4, g4), 5) * 1e3,
                "disc_ms_per_call": _time_calls(lambda: ctx.discriminant_res(f4), 5) * 1e3,
                "primes": {"res": api.resultant_info(f4, g4)["primes"],
                           "disc": api.resultant_info(f4, None, disc=True)["primes"]},
                "oracle_res_s": per["c4_res"][0],
                "workload": "product of 8 circles/ellipses + 16 monomials (32-bit) vs dense degree 24, 64-bit "
                            "(seed 4)"}
    # 5: serving
    if serve_requests > 0:
        out["5"] = serving_loads(ctx, serve_requests)
        out["5"]["oracle"] = oracle_rate("c5")
    return out


# --------------------------------------------------------------------------- our arm


def traffic_for() -> float | None:
    """Per-launch DRAM bytes of the evaluation kernel from the committed ncu summary,
    if that summary describes the current kernel source (the hash of its source
    files, in the order the summary lists them)."""
    path = os.path.join(ROOT, "profiles", "evalres_dram.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    files = d.get("source_files") or []
    if not files or not all(os.path.exists(os.path.join(ROOT, f)) for f in files):
        return None
    h = hashlib.sha256(b"".join(open(os.path.join(ROOT, f), "rb").read() for f in files)).hexdigest()[:16]
    return d.get("bytes_per_launch_full") if d.get("source_sha") == h else None


def run_ours(args) -> None:
    import torch

    import oracle as O
    from paper_1103_4697_gb300 import api
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_baseline()          # spawn pool: safe before or after CUDA init
    ctx = api.Context(device=local, mem_budget=args.mem_gb << 30)
    cal = ctx.calibrate()
    NP = args.pairs
    base = rank_seed_base(rank, NP)
    F, G = W.deg20_batch_arrays(NP, base, DEG, BITS)
    res = ctx.upload_pairs(F, G)
    ctx.set_option(N.OPT_STATS, 1)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    for _ in range(args.warmup):
        res.run()
    # parity spot check (outside the timed region): 8 pairs drawn from the whole batch,
    # each at two random points against the oracle's exact R(a)
    rng = random.Random(rank)
    spot = rng.sample(range(NP), min(8, NP))
    for q in spot:
        out = res.fetch(q, 1)[0]
        for a in (rng.randint(-2 ** 31, 2 ** 31), rng.randint(-2 ** 31, 2 ** 31)):
            v = 0
            for c in reversed(out):
                v = v * a + c
            assert v == O.res_at_prs(F[q], G[q], a), f"parity spot check failed (pair {q}, x = {a})"
    clocks = ClockSampler(local)
    evs = []
    stage = {k: 0.0 for k in ("bounds_ms", "reduce_ms", "evalres_ms", "interp_ms", "crt_ms")}
    kernels = 0
    st = {}
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)                                  # evict L2 between steps (untimed)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        res.run()
        e.record(stream)
        evs.append((s, e))
        st = ctx.stats()
        for k in stage:
            stage[k] += st[k]
        kernels += st["kernels"]
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier(world)
    clk = clocks.stop()
    dev_ms = sum(s.elapsed_time(e) for s, e in evs)
    dev_ms = reduce_max(dev_ms, world)
    value = world * NP * args.steps / (dev_ms * 1e-3)
    evalres_ms = stage["evalres_ms"] / args.steps
    # roofline of the dominant stage: the modular products its code executes per
    # launch, against the rate this GPU reaches for the same mix of operations
    # (each kind at its calibrated rate)
    plans = res.plan()
    quartic = st["quad_pairs"] == NP            # the point set the planner chose
    rl = evalres_roofline(F, G, plans, api.primes(max(p["primes"] for p in plans)), cal, quartic)
    achieved = rl["products"] / (evalres_ms * 1e-3)
    peak = rl["products"] / rl["ideal_s"]
    best_single = max(cal["modmul_per_s"], 2 * cal["mulsub_per_s"], 3 * cal["fma3_per_s"], cal["shoup_per_s"])
    # e2e: the public C call with host buffers (H2D of inputs and D2H of results inside)
    keep = api._Packed()
    df, dg = api.pack_bipolys(F, keep), api.pack_bipolys(G, keep)
    outs = (N.BigPoly * NP)()
    L = N.lib()
    e2e_steps = max(2, min(args.steps, 6))
    # untimed warm-up calls, as for the device-timed steps (the first call builds the
    # one-shot batch cache and the pipeline workers)
    for _ in range(max(1, args.warmup)):
        N.check(L.gbr_resultant_batch(ctx.handle, NP, api._ptr(df), api._ptr(dg), 1, outs), ctx.handle)
        for i in range(NP):
            L.gbr_free_result(ctx.handle, C.byref(outs[i]))
    torch.cuda.synchronize()
    t = time.perf_counter()
    h2d = d2h = 0
    for _ in range(e2e_steps):
        N.check(L.gbr_resultant_batch(ctx.handle, NP, api._ptr(df), api._ptr(dg), 1, outs), ctx.handle)
        s2 = ctx.stats()
        h2d, d2h = s2["h2d_bytes"], s2["d2h_bytes"]
        t_free = time.perf_counter()
        for i in range(NP):
            L.gbr_free_result(ctx.handle, C.byref(outs[i]))
        t += time.perf_counter() - t_free           # freeing the returned buffers is not timed
    e2e_s = reduce_max(time.perf_counter() - t, world)
    e2e = {"value": world * NP * e2e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "api": "gbr_resultant_batch (host buffers)"}
    # the plain GPU path: one pair per call
    one = None
    configs = None
    if rank == 0:
        n1 = 64
        t = time.perf_counter()
        for q in range(n1):
            o = N.BigPoly()
            N.check(L.gbr_resultant(ctx.handle, C.cast(api._ptr(df[q:q + 1]), C.POINTER(N.BiPoly)),
                                    C.cast(api._ptr(dg[q:q + 1]), C.POINTER(N.BiPoly)), 1, C.byref(o)), ctx.handle)
            L.gbr_free_result(ctx.handle, C.byref(o))
        one = {"value": n1 / (time.perf_counter() - t), "unit": "solves/s", "sample": f"{n1} pairs, one call each"}
        if not args.no_configs:
            res.free()
            res = None
            configs = configs_block(ctx, cal, 0 if args.no_serve else args.serve_requests)
    if res is not None:
        res.free()
    ctx.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{NP} dense pairs (f, g), total degree {DEG}, {BITS}-bit signed coefficients, "
                               f"seeds {BASE_SEED}+i per pair (+{NP}*rank)", "pairs_per_gpu": NP,
                   "degree": DEG, "coef_bits": BITS, "inputs": "device-resident", "l2": "flushed between steps "
                   "(256 MiB write)", "parallelism": "replicas" if world > 1 else "single GPU"},
        "clocks": clk, "e2e": e2e, "gpu_launches": kernels,
        "roofline": {"bound": "alu", "kernel": "k_evalres_reg<20> (+ k_evalres_redo)", "achieved": achieved / 1e12,
                     "peak": peak / 1e12, "unit": "Tmodmul/s", "frac": achieved / peak, "traffic": traffic_for(),
                     "peak_source": "measured on this GPU by gbr_calibrate (independent chains): the kernel's own "
                                    "mix of Shoup Horner steps, Montgomery products, fused 2- and 3-product "
                                    "reductions, each at its calibrated rate",
                     "products_per_launch": rl["products"], "ops_per_launch": rl["ops"],
                     "textbook_products_per_launch": rl["textbook_products"],
                     "frac_of_best_single_form": achieved / best_single,
                     "points": plans[0]["deg_bound"] + 1,
                     "point_set": "quartic 0, +-a, +-i a (radix-4 evaluation)" if quartic else "symmetric integers",
                     "primes": [min(p["primes"] for p in plans), max(p["primes"] for p in plans)]},
        "cpu_baseline": cpu,
        "stages_ms": {k: v / args.steps for k, v in stage.items()},
        "wall_ms_per_step": t_wall * 1e3 / args.steps,
        "calibration": cal,
        "one_pair_per_launch": one,
        "configs": configs,
        "serving": (configs or {}).get("5"),
        "parity": "8 pairs drawn from the whole batch x 2 random points vs the oracle's R(a) before timing; "
                  "every pair in tests -m gpu",
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------- reference arm


def run_reference(args) -> None:
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    per = []
    t_all = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = oracle_baseline(1, cores)
        per.append(last["value"])
    wall = time.perf_counter() - t_all
    value = statistics.mean(per)
    line = {
        "metric": METRIC, "impl": "reference", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int (arbitrary precision)",
        "data": "synthetic",
        "config": {"workload": f"{PAIRS} dense pairs (f, g), total degree {DEG}, {BITS}-bit signed coefficients, "
                               f"seeds {BASE_SEED}+i; each step a bounded sample of {cores} pairs",
                   "pairs_per_gpu": PAIRS, "degree": DEG, "coef_bits": BITS},
        "cpu_baseline": dict(last, value=value),
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------- other workloads


def _time_calls(fn, reps: int) -> float:
    import torch

    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t) / reps


def _oracle_time(fn, *a) -> float:
    t = time.perf_counter()
    fn(*a)
    return time.perf_counter() - t


def ntt_crossover(ctx, reps: int = 5) -> dict:
    """Integer points (inverse-Vandermonde contraction or Newton) against roots of unity
    (inverse transform) on batches of one shape each, x-degree bound D from 64 to 16 380:
    device time per run (CUDA events around the resident run, median of `reps`), the
    evaluation and interpolation stages, and what the automatic choice takes."""
    import torch

    from paper_1103_4697_gb300 import native as N

    def pair(rng, m, dx, bits=12):
        h = 1 << (bits - 1)
        f = [[rng.randint(-h, h - 1) for _ in range(dx + 1)] for _ in range(m + 1)]
        f[-1][-1] = f[-1][-1] or 1
        return f

    shapes = [(2, dx) for dx in (16, 32, 64, 100, 128, 200, 256, 512, 1024, 2048, 4095)]
    shapes += [(8, dx) for dx in (8, 16, 32, 64, 128, 256, 512)]
    shapes += [("dense", d) for d in (8, 12, 16, 20, 24)] + [("mixed", 4096)]
    rows = []
    stream = torch.cuda.current_stream()
    ctx.set_option(N.OPT_STATS, 1)
    for m, dx in shapes:
        rng = random.Random(hash((m, dx)) & 0xffff)
        from paper_1103_4697_gb300 import workloads as W
        if m == "dense":
            F, G = W.deg20_batch_arrays(1024, 5000 + dx, dx, 16)
            fs, gs, label, D = F, G, f"dense total degree {dx}", dx * dx
        elif m == "mixed":
            ps = W.mixed_batch(3, dx)
            fs, gs, label, D = ps.f, ps.g, "heterogeneous batch (degrees 4..16, 25% planted)", 512
        else:
            npairs = max(8, min(1024, 4_000_000 // (2 * m * dx * (m + 1) * (dx + 1))))
            fs = [pair(rng, m, dx) for _ in range(npairs)]
            gs = [pair(rng, m, dx) for _ in range(npairs)]
            label, D = f"y-degree {m}, x-degree {dx}", 2 * m * dx
        res = ctx.upload_pairs(fs, gs)
        row = {"shape": label, "pairs": len(fs), "D": D}
        outs = {}
        for mode, name in ((1, "integer"), (2, "roots"), (0, "auto")):
            ctx.set_option(N.OPT_POINTS, mode)
            for _ in range(2):
                res.run()
            times = []
            for _ in range(reps):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(stream)
                res.run()
                e.record(stream)
                e.synchronize()
                times.append(s.elapsed_time(e))
            st = ctx.stats()
            outs[name] = res.fetch(0, min(4, len(fs)))
            row[name] = {"us_per_pair": statistics.median(times) * 1e3 / len(fs),
                         "stages_ms": {k: round(st[k], 4) for k in ("bounds_ms", "reduce_ms", "evalres_ms",
                                                                     "interp_ms", "crt_ms")},
                         "root_pairs": st["root_pairs"]}
        assert outs["integer"] == outs["roots"] == outs["auto"], label
        row["auto_picks"] = "roots" if row["auto"]["root_pairs"] else "integer"
        row["faster"] = "roots" if row["roots"]["us_per_pair"] < row["integer"]["us_per_pair"] else "integer"
        res.free()
        rows.append(row)
    ctx.set_option(N.OPT_POINTS, 0)
    return {"ntt_crossover": rows,
            "workload": "batches of random pairs per shape (12-bit coefficients; dense rows: 16-bit), "
                        "integer points vs roots of unity vs automatic choice"}


def run_config(args) -> None:
    """Measurements for the other workloads (one JSON line each):
    small   one dense degree-6 pair, res_y and gcd(f(x,0), g(x,0)), one call each;
    deg20   one degree-20 pair, res_y(f, g) and res_y(f, f_y), one call each;
    mixed   4096 mixed pairs (degrees 4..16, 8..32-bit, 25 % planted), resident batch,
            and 4096 gcd jobs (degrees 30..200, planted degree-5 factor);
    conic   product of 8 conics (+ sparse terms) against a dense degree-24 curve with
            64-bit coefficients: res_y(f, g) and res_y(f, f_y), one call each;
    serve   Poisson streams of mixed requests at 0.5, 0.8 and 0.95 of the measured capacity;
    gcd     the 4096 gcd jobs alone, through the C ABI with packed host buffers;
    arrangement  the n(n+1)/2 resultants of an arrangement of 90 curves (Section 3:
            res(f, f_y) per curve, res(f, g) per pair; 4095 jobs) in one pass, then the
            square-free factorisation of all of them (Section 2.1);
    teissier  the Teissier resultant Q = res(f_x/h, f_y/h, y), h = gcd(f_x, f_y)
            (Section 2.1), for 1024 curves shaped like the arrangement's (degree 8);
    sqf     square-free factorisation R = u prod r_i^i (Section 2.1) of 2048 planted
            projection-resultant-shaped polynomials, through the C ABI, and of
            R = res_y(f, f_y) of the conic-product curve (the path's own output)."""
    import torch

    import oracle as O
    from paper_1103_4697_gb300 import api
    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300 import workloads as W

    torch.cuda.set_device(0)
    ctx = api.Context(device=0, mem_budget=args.mem_gb << 30)
    out = {"config": args.config, "data": "synthetic", "n_gpus": 1}
    if args.config == "small":
        f, g = W.small_dense_pair(1)
        p, q = list(f[0]), list(g[0])
        ctx.resultant(f, g)
        ctx.gcd(p, q)
        out["res_ms"] = _time_calls(lambda: ctx.resultant(f, g), 20) * 1e3
        out["gcd_ms"] = _time_calls(lambda: ctx.gcd(p, q), 20) * 1e3
        out["oracle_res_ms"] = _oracle_time(O.res_bareiss, f, g) * 1e3
        out["oracle_gcd_ms"] = _oracle_time(O.gcd_z, p, q) * 1e3
        out["workload"] = "dense total degree 6, coefficients in [-128, 127] (seed 1)"
    elif args.config == "deg20":
        f, g = W.deg20_pair(2)
        ctx.resultant(f, g)
        out["res_ms"] = _time_calls(lambda: ctx.resultant(f, g), 10) * 1e3
        out["disc_ms"] = _time_calls(lambda: ctx.discriminant_res(f), 10) * 1e3
        out["oracle_res_ms"] = _oracle_time(O.res_evalz, f, g) * 1e3
        out["oracle_disc_ms"] = _oracle_time(O.disc_res, f, "evalz") * 1e3
        out["workload"] = "dense total degree 20, 16-bit (seed 2), one call per resultant"
    elif args.config == "conic":
        f, g = W.conic_curves(4)
        info = api.resultant_info(f, g)
        dinfo = api.resultant_info(f, None, disc=True)
        ctx.resultant(f, g)
        out["res_ms"] = _time_calls(lambda: ctx.resultant(f, g), 5) * 1e3
        out["disc_ms"] = _time_calls(lambda: ctx.discriminant_res(f), 5) * 1e3
        out["primes"] = {"res": info["primes"], "disc": dinfo["primes"]}
        out["oracle_res_ms"] = _oracle_time(O.res_evalz, f, g) * 1e3
        out["workload"] = "8 conics + 16 monomials (32-bit) vs dense degree 24, 64-bit (seed 4)"
    elif args.config == "mixed":
        ps = W.mixed_batch(3, PAIRS)
        ctx.set_option(N.OPT_STATS, 1)
        res = ctx.upload_pairs(ps.f, ps.g)
        for _ in range(5):  # from the fourth run on the whole step replays from its graph
            res.run()
        st0 = ctx.stats()
        sec = _time_calls(res.run, 10)
        outs = res.fetch()
        assert all(outs[i] == [] for i in range(PAIRS) if ps.planted[i])
        res.free()
        out["res_solves_per_s"] = PAIRS / sec
        out["res_stages_ms"] = {k: st0[k] for k in ("bounds_ms", "reduce_ms", "evalres_ms", "interp_ms", "crt_ms")}
        P, Q, H = W.gcd_batch(3, PAIRS)
        got = ctx.gcd_batch(P, Q)
        gsec = _time_calls(lambda: ctx.gcd_batch(P, Q), 3)
        out["gcd_jobs_per_s_python_lists"] = PAIRS / gsec
        # through the C ABI with packed host buffers (what a native caller pays):
        # copies, kernels and the certificate; freeing the results is not timed
        keep = api._Packed()
        dp, dq = api.pack_upolys(P, keep), api.pack_upolys(Q, keep)
        L = N.lib()
        gouts = (N.BigPoly * PAIRS)()
        t_gcd = 0.0
        for _ in range(5):
            t0 = time.perf_counter()
            N.check(L.gbr_gcd_batch(ctx.handle, PAIRS, api._ptr(dp), api._ptr(dq), gouts), ctx.handle)
            t_gcd += time.perf_counter() - t0
            gst = ctx.stats()
            for i in range(PAIRS):
                L.gbr_free_result(ctx.handle, C.byref(gouts[i]))
        out["gcd_jobs_per_s"] = 5 * PAIRS / t_gcd
        out["gcd_stats"] = {k: gst[k] for k in ("gcd_ms", "total_ms", "kernels", "subproblems", "h2d_bytes",
                                                "d2h_bytes")}
        assert all(len(got[i]) - 1 >= 5 for i in range(0, PAIRS, 97))   # the planted degree-5 factor divides
        t = time.perf_counter()
        for i in range(4):
            O.res_evalz(ps.f[i], ps.g[i])
        out["oracle_res_solves_per_s_1core"] = 4 / (time.perf_counter() - t)
        t = time.perf_counter()
        for i in range(4):
            O.gcd_z(P[i], Q[i])
        out["oracle_gcd_jobs_per_s_1core"] = 4 / (time.perf_counter() - t)
        out["workload"] = "4096 pairs deg_x, deg_y ~ U{4..16}, 8..32-bit, 25% planted (seed 3); 4096 gcds deg 30..200"
    elif args.config == "gcd":
        # the gcd batch alone, through the C ABI with packed host buffers
        P, Q, H = W.gcd_batch(3, PAIRS)
        keep = api._Packed()
        dp, dq = api.pack_upolys(P, keep), api.pack_upolys(Q, keep)
        ctx.set_option(N.OPT_STATS, 1)
        L = N.lib()
        gouts = (N.BigPoly * PAIRS)()
        times = []
        for it in range(6):
            t0 = time.perf_counter()
            N.check(L.gbr_gcd_batch(ctx.handle, PAIRS, api._ptr(dp), api._ptr(dq), gouts), ctx.handle)
            times.append(time.perf_counter() - t0)
            gst = ctx.stats()
            for i in range(PAIRS):
                L.gbr_free_result(ctx.handle, C.byref(gouts[i]))
        sec = statistics.median(times[1:])
        out["gcd_jobs_per_s"] = PAIRS / sec
        out["gcd_stats"] = {k: gst[k] for k in ("gcd_ms", "total_ms", "kernels", "subproblems", "h2d_bytes",
                                                "d2h_bytes")}
        out["workload"] = "4096 gcds deg 30..200, planted degree-5 factor, 8..32-bit cofactors (seed 3)"
    elif args.config == "arrangement":
        NC = 90
        curves = W.arrangement_curves(7, n=NC, d=8, bits=12, conic_frac=0.25, rbits=6)
        NJ = NC * (NC + 1) // 2
        keep = api._Packed()
        df = api.pack_bipolys(curves, keep)
        ctx.set_option(N.OPT_STATS, 1)
        L = N.lib()
        outs = (N.BigPoly * NJ)()
        times = []
        for it in range(6):
            t0 = time.perf_counter()
            N.check(L.gbr_arrangement_resultants(ctx.handle, NC, api._ptr(df), 1, outs), ctx.handle)
            times.append(time.perf_counter() - t0)
            if it < 5:
                for i in range(NJ):
                    L.gbr_free_result(ctx.handle, C.byref(outs[i]))
        sec = statistics.median(times[1:])
        allres = ctx._collect(outs, NJ)
        out["arrangement_jobs_per_s_e2e"] = NJ / sec
        out["arrangement_ms_per_call"] = sec * 1e3
        res = ctx.upload_arrangement(curves)
        for _ in range(3):
            res.run()
        rt = []
        for _ in range(10):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res.run()
            rt.append(time.perf_counter() - t0)
        st = ctx.stats()
        res.free()
        out["arrangement_jobs_per_s_resident"] = NJ / statistics.median(rt)
        out["resident_stages_ms"] = {k: st[k] for k in ("bounds_ms", "reduce_ms", "evalres_ms", "interp_ms", "crt_ms")}
        # projection phase: square-free factorisation of every resultant of the arrangement
        sk = api._Packed()
        arr = api.pack_bigpolys(allres, sk)
        souts = (N.Sqf * NJ)()
        stimes = []
        for it in range(4):
            t0 = time.perf_counter()
            N.check(L.gbr_squarefree_batch(ctx.handle, NJ, arr, souts), ctx.handle)
            stimes.append(time.perf_counter() - t0)
            counts = [souts[i].count for i in range(NJ)]
            for i in range(NJ):
                L.gbr_free_sqf(ctx.handle, C.byref(souts[i]))
        out["sqf_of_all_ms"] = statistics.median(stimes[1:]) * 1e3
        out["resultants_with_repeated_factors"] = sum(1 for k in counts if k >= 2)
        degs = [len(r) - 1 for r in allres]
        bits = [max(abs(c) for c in r).bit_length() if r else 0 for r in allres]
        out["result_degree_max"] = max(degs)
        out["result_bits_max"] = max(bits)
        t = time.perf_counter()
        O.res_subres(curves[0], curves[1])
        O.disc_res(curves[2])
        out["oracle_jobs_per_s_1core"] = 2 / (time.perf_counter() - t)
        out["workload"] = ("arrangement of 90 curves (seed 7): 25% products of 4 circles/ellipses (radii/centres "
                           "in [-64, 64]), 75% dense total degree 8 with 12-bit coefficients; 90 res(f, f_y) + "
                           "4005 res(f, g) per pass")
    elif args.config == "teissier":
        NT = 1024
        curves = W.arrangement_curves(11, n=NT, d=8, bits=12, conic_frac=0.25, rbits=4)
        keep = api._Packed()
        df = api.pack_bipolys(curves, keep)
        L = N.lib()
        outs = (N.BigPoly * NT)()
        times = []
        for it in range(5):
            t0 = time.perf_counter()
            N.check(L.gbr_teissier_res_batch(ctx.handle, NT, api._ptr(df), outs), ctx.handle)
            times.append(time.perf_counter() - t0)
            got = ctx._collect(outs, NT)
        sec = statistics.median(times[1:])
        out["teissier_jobs_per_s"] = NT / sec
        out["teissier_ms_per_call"] = sec * 1e3
        out["q_degree_max"] = max(len(q) - 1 for q in got)
        for k in random.Random(3).sample(range(NT), 2):      # parity spot check before reporting
            assert got[k] == list(O.teissier_q(curves[k])), k
        t = time.perf_counter()
        for k in range(2):
            O.teissier_q(curves[k])
        out["oracle_teissier_jobs_per_s_1core"] = 2 / (time.perf_counter() - t)
        out["workload"] = ("Q = res(f_x/h, f_y/h, y) for 1024 curves (seed 11): 25% products of 4 circles/ellipses "
                           "(centres and radii in [-16, 16]), 75% dense total degree 8, 12-bit")
    elif args.config == "sqf":
        NS = 2048
        R, _ = W.sqf_batch(6, NS)
        keep = api._Packed()
        arr = api.pack_bigpolys(R, keep)
        ctx.set_option(N.OPT_STATS, 1)
        L = N.lib()
        souts = (N.Sqf * NS)()
        times = []
        for it in range(6):
            t0 = time.perf_counter()
            N.check(L.gbr_squarefree_batch(ctx.handle, NS, arr, souts), ctx.handle)
            times.append(time.perf_counter() - t0)
            sst = ctx.stats()
            for i in range(NS):
                L.gbr_free_sqf(ctx.handle, C.byref(souts[i]))
        sec = statistics.median(times[1:])
        out["sqf_jobs_per_s"] = NS / sec
        out["sqf_ms_per_call"] = sec * 1e3
        out["sqf_stats"] = {k: sst[k] for k in ("gcd_ms", "total_ms", "kernels", "subproblems", "h2d_bytes",
                                                "d2h_bytes")}
        t = time.perf_counter()
        for i in range(4):
            O.sqf_yun(R[i])
        out["oracle_sqf_jobs_per_s_1core"] = 4 / (time.perf_counter() - t)
        # the paper's chain: R = res_y(f, f_y) of a product of 8 circles/ellipses
        # (singular at their intersections, so R has squared factors), then Yun on R
        f, _g = W.conic_curves(4, nterms=0)
        Rc = ctx.discriminant_res(f)
        ctx.squarefree(Rc)
        tc = _time_calls(lambda: ctx.squarefree(Rc), 5)
        u, facs = ctx.squarefree(Rc)
        out["conic_R"] = {"deg": len(Rc) - 1, "max_bits": max(abs(c).bit_length() for c in Rc),
                          "factor_degrees": [len(x) - 1 for x in facs], "sqf_ms": tc * 1e3}
        out["workload"] = ("2048 R = u r1 r2^2 r3^3, deg r_i ~ U{20..60}, U{4..16}, U{0..4}, 16-bit "
                           "(deg R 28..104, about 100-bit coefficients; seed 6); R = res_y(f, f_y) of 8 conics (seed 4)")
    elif args.config == "ntt":
        out.update(ntt_crossover(ctx))
    elif args.config == "serve":
        res_all = {}
        cap = None
        for load in (0.5, 0.8, 0.95):
            r = serving_run(ctx, n_burst=3000, n_stream=args.serve_requests, load=load, seed=5, capacity=cap)
            cap = r["capacity_rps"]
            res_all[str(load)] = {k: r[k] for k in ("p50_ms", "p99_ms", "throughput_rps", "offered_rps")}
        out["capacity_rps"] = cap
        out["loads"] = res_all
        out["workload"] = (f"{args.serve_requests} Poisson-arrival requests per load, 50/50 res_y/gcd, degree "
                           "log-uniform 5..30, 8..64-bit, 10% planted (seed 5)")
    ctx.close()
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mem-gb", type=int, default=24)
    ap.add_argument("--pairs", type=int, default=PAIRS, help="pairs per GPU (smaller only for profiling)")
    ap.add_argument("--config", choices=["headline", "small", "deg20", "mixed", "conic", "serve", "gcd", "sqf",
                                                 "arrangement", "teissier", "ntt"],
                    default="headline", help="other workloads print their own JSON line")
    ap.add_argument("--serve-requests", type=int, default=100_000,
                    help="requests per load of the serving configuration (default: its stated 100 000)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="headline line without the per-configuration block")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.config != "headline":
        run_config(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
