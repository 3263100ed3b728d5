"""Host-side native code on the CPU (no GPU): the big-integer routines of the
square-free path (Knuth's long division, Lehmer's gcd, gcd_into) checked against
Python integers on seeded random operands, and the host worker pool behind
gbr_parallel_for under concurrent and nested use.  The C++ harnesses live in
tests/native/ and are compiled here with g++.
"""

import math
import os
import shutil
import subprocess

import pytest

from paper_1103_4697_gb300 import native as N

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _gxx():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    return gxx


def _build(tmp_path, src, extra=()):
    exe = str(tmp_path / os.path.splitext(os.path.basename(src))[0])
    cmd = [_gxx(), "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "native", src), *extra]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def _int(line):
    t = [int(v) for v in line.split()]
    return sum(v << (32 * k) for k, v in enumerate(t[1:1 + t[0]]))


def test_bigint_division_and_gcd_match_python(tmp_path):
    exe = _build(tmp_path, "bigint_harness.cpp")
    out = subprocess.run([exe, "1500"], check=True, capture_output=True, text=True).stdout.split("\n")
    n = int(out[0])
    i, bad = 1, []
    for case in range(n):
        a, b, q, r, g1, g2 = (_int(out[i + k]) for k in range(6))
        i += 6
        if (q, r) != divmod(a, b) or g1 != math.gcd(a, b) or g2 != math.gcd(a, b):
            bad.append(case)
    assert n == 1500 and not bad, bad[:10]


def test_host_pool_visits_every_index_once(tmp_path):
    if not os.path.exists(N.LIB_PATH):
        from paper_1103_4697_gb300.build import build

        build()
    libdir = os.path.dirname(N.LIB_PATH)
    extra = [f"-L{libdir}", "-lgbres", f"-Wl,-rpath,{libdir}", "-pthread"]
    cuda_lib = "/usr/local/cuda/lib64"
    if os.path.isdir(cuda_lib):
        extra += [f"-L{cuda_lib}", f"-Wl,-rpath,{cuda_lib}"]
    exe = _build(tmp_path, "pool_harness.cpp", extra)
    res = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120)
    assert res.stdout.strip() == "bad 0", res.stdout


def _signed(line, L):
    t = [int(v) for v in line.split()]
    return t[0] * sum(v << (32 * k) for k, v in enumerate(t[1:1 + L]))


def test_sqf_primitive_parts_and_norms(tmp_path):
    """primitive_part returns the primitive part with a positive leading coefficient
    (contents of up to three limbs planted); the norms are upper bounds of the exact
    log2 norms within 1e-6 bit."""
    exe = _build(tmp_path, "sqf_host_harness.cpp")
    out = subprocess.run([exe, "1000"], check=True, capture_output=True, text=True).stdout.split("\n")
    n, i = int(out[0]), 1
    bad, loose = [], []
    for case in range(n):
        d, L = map(int, out[i].split())
        i += 1
        c = [_signed(out[i + t], L) for t in range(d + 1)]
        i += d + 1
        ok, FL = map(int, out[i].split())
        i += 1
        g = 0
        for v in c:
            g = math.gcd(g, v)
        want = [v // g * (1 if c[-1] > 0 else -1) for v in c]
        if not ok:
            bad.append(case)
        else:
            got = [_signed(out[i + t], FL) for t in range(d + 1)]
            i += d + 1
            if got != want:
                bad.append(case)
        l1, l2, li = map(float, out[i].split())
        i += 1
        e1 = math.log2(sum(abs(v) for v in c))
        e2 = 0.5 * math.log2(sum(v * v for v in c))
        ei = math.log2(max(abs(v) for v in c))
        if not (e1 <= l1 <= e1 + 1e-6 and e2 <= l2 <= e2 + 1e-6 and ei <= li <= ei + 1e-6):
            loose.append(case)
    assert n == 1000 and not bad and not loose, (bad[:5], loose[:5])
