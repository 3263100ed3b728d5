"""Host-side tests of libgbres (no GPU): the library loads, exports every entry
point include/gbres.h declares, and its host-only planning (prime table, prime
counts, degree and coefficient bounds) is right."""

import ctypes as C
import math
import os
import random
import re

import pytest

import oracle as O
from paper_1103_4697_gb300 import native as N
from paper_1103_4697_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(N.LIB_PATH):
        from paper_1103_4697_gb300.build import build
        build()
    return N.lib()


def _header_functions():
    text = open(os.path.join(ROOT, "include", "gbres.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbr_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(N.SIGNATURES) == names
    assert N.missing_symbols() == []


def _is_prime(n):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def test_prime_table(lib):
    from paper_1103_4697_gb300.api import primes

    assert lib.gbr_num_primes() == 2048
    ps = primes(2048)
    step = 1 << 14
    # the largest primes below 2^32 / 3 that are 1 mod 2^14 (roots of unity of order 2^14)
    assert ps[0] < 2 ** 32 // 3 and not any(_is_prime(c) for c in range(ps[0] + step, 2 ** 32 // 3 + 1, step))
    assert all(a > b for a, b in zip(ps, ps[1:]))
    assert all(p % step == 1 for p in ps) and ps[-1] > 2 ** 30
    assert all(_is_prime(p) for p in ps[:300] + ps[-20:])
    # consecutive: no such prime is skipped between table entries
    for a, b in zip(ps[:40], ps[1:41]):
        assert not any(_is_prime(c) for c in range(b + step, a, step))
    p = C.c_uint32()
    assert lib.gbr_prime(2048, C.byref(p)) == N.EINVAL
    assert lib.gbr_prime(-1, C.byref(p)) == N.EINVAL


def test_reduction_shoup_constant(lib):
    """The reduction kernel forms c R^2 mod p (R = 2^32) of a one-word coefficient by one
    Shoup product with W = R^2 mod p, taking floor(W 2^32 / p) as (R^3 mod p) times
    -p^-1 modulo 2^32 (W 2^32 = floor(W 2^32 / p) p + (R^3 mod p), an exact division).
    For every 32-bit c the product c W - floor(c W' / 2^32) p lies in [0, 2p)."""
    from paper_1103_4697_gb300.api import primes

    R = 1 << 32
    rng = random.Random(5)
    for p in primes(64):
        W, t3 = R * R % p, R ** 3 % p
        wp = t3 * ((-pow(p, -1, R)) % R) % R
        assert wp == W * R // p
        for c in [0, 1, p - 1, p, p + 1, 2 ** 31, R - 1] + [rng.randrange(R) for _ in range(100)]:
            r = (c * W - ((c * wp) >> 32) * p) % R
            assert r < 2 * p and r % p == c * W % p


@pytest.mark.parametrize("bits", [0.0, 1.0, 30.0, 31.0, 61.9, 100.0, 860.0, 9500.0])
def test_primes_for_bits(lib, bits):
    from paper_1103_4697_gb300.api import primes

    k = lib.gbr_primes_for_bits(bits)
    ps = primes(k)
    assert sum(math.log2(p) for p in ps) > bits
    assert k == 1 or sum(math.log2(p) for p in ps[:-1]) <= bits + 1e-5


@pytest.mark.parametrize("seed", range(12))
def test_resultant_info_bounds(lib, seed):
    """Degrees match the oracle's, the x-degree bound holds, and every coefficient of
    the exact resultant is below 2^log2_bound (Hadamard)."""
    from paper_1103_4697_gb300.api import resultant_info

    rng = random.Random(seed)
    d = rng.randint(1, 6)
    f, g = W.small_dense_pair(900 + seed, d, rng.randint(2, 20))
    info = resultant_info(f, g)
    assert (info["m"], info["n"]) == (O.ydeg(f), O.ydeg(g))
    R = O.res_subres(f, g)
    assert len(R) - 1 <= info["deg_bound"]
    assert info["deg_bound"] <= d * d
    for c in R:
        assert abs(c) == 0 or math.log2(abs(c)) <= info["log2_bound"] + 1e-9
    prod = 1
    from paper_1103_4697_gb300.api import primes
    for p in primes(info["primes"]):
        prod *= p
    assert all(prod > 2 * abs(c) + 1 for c in R)
    di = resultant_info(f, None, disc=True)
    Rd = O.disc_res(f)
    assert di["n"] == O.ydeg(f) - 1
    assert len(Rd) - 1 <= di["deg_bound"]
    assert all(abs(c) == 0 or math.log2(abs(c)) <= di["log2_bound"] + 1e-9 for c in Rd)


def test_resultant_info_var0_and_zero(lib):
    from paper_1103_4697_gb300.api import resultant_info

    f = [[1, 2, 3], [4, 5, 0]]        # deg_y 1, deg_x 2
    g = [[1, 1], [0, 2], [3, 0]]      # deg_y 2, deg_x 1
    i1 = resultant_info(f, g, var=0)
    assert (i1["m"], i1["n"]) == (2, 1)
    z = resultant_info([[0, 0]], g)
    assert z["m"] == -1


def test_status_strings_and_bad_create(lib):
    assert lib.gbr_strerror(N.OK) == b"ok"
    assert lib.gbr_strerror(N.ENOMEM).startswith(b"out of memory")
    h = C.c_void_p()
    assert lib.gbr_create(C.byref(h), 0, 1000, None, None) == N.EINVAL   # budget below 1 MiB
    assert lib.gbr_create(None, 0, 1 << 30, None, None) == N.EINVAL


@pytest.mark.parametrize("seed", range(40))
def test_scaled_bound_holds_on_varied_shapes(lib, seed):
    """The planner's bound (minimum of row/column Hadamard bounds over scalings y ->
    lambda y) is at least the true size of every coefficient, for dense boxes,
    total-degree polynomials, sparse polynomials with large leading coefficients and
    products with planted roots."""
    from paper_1103_4697_gb300.api import resultant_info

    rng = random.Random(1000 + seed)
    kind = seed % 4
    if kind == 0:
        f, g = W.small_dense_pair(seed, rng.randint(1, 7), rng.randint(2, 30))
    elif kind == 1:
        f = W.dense_box(W.Stream(seed), rng.randint(0, 5), rng.randint(1, 6), rng.randint(2, 40))
        g = W.dense_box(W.Stream(seed + 99), rng.randint(0, 5), rng.randint(1, 6), rng.randint(2, 40))
    elif kind == 2:
        m, n = rng.randint(1, 6), rng.randint(1, 6)
        f = [[0] * 4 for _ in range(m + 1)]
        g = [[0] * 4 for _ in range(n + 1)]
        f[m][rng.randint(0, 3)] = rng.choice([-1, 1]) * rng.randint(1, 2 ** 40)
        g[n][rng.randint(0, 3)] = rng.choice([-1, 1]) * rng.randint(1, 2 ** 40)
        for _ in range(4):
            f[rng.randint(0, m)][rng.randint(0, 3)] = rng.randint(-2 ** 20, 2 ** 20)
            g[rng.randint(0, n)][rng.randint(0, 3)] = rng.randint(-2 ** 20, 2 ** 20)
    else:
        f, g, *_ = W.planted_roots_pair(seed, rng.randint(1, 5), rng.randint(1, 5), bits=rng.randint(2, 12))
    if O.ydeg(f) < 0 or O.ydeg(g) < 0:
        return
    for disc in (False, True):
        info = resultant_info(f, None if disc else g, disc=disc)
        R = O.disc_res(f) if disc else O.res_subres(f, g)
        if info["m"] < 0 or info["n"] < 0:
            assert R == ()
            continue
        assert all(c == 0 or math.log2(abs(c)) <= info["log2_bound"] + 1e-9 for c in R), (info, disc)
        assert len(R) - 1 <= info["deg_bound"]


def _rand_rows(rng, dy, dx, amp):
    rows = [[rng.randint(-amp, amp) for _ in range(dx + 1)] for _ in range(dy + 1)]
    rows[dy][dx] = amp                                   # full degree in both variables
    return rows


def test_resultant_info_at_the_size_limits(lib):
    """The documented limits of include/gbres.h on the host-side plan: y-degree
    GBR_MAX_YDEG (127) and 8-word (511-bit) coefficients are planned, y-degree 128
    and a 512-bit coefficient (9 words) are refused with GBR_ELIMIT and GBR_EINVAL.
    The 8-word pair of y-degree 56 needs between 1321 and 2048 primes, so its
    result is wider than 1280 limbs (the Chinese remaindering's narrow-block case);
    y-degree 64 needs more than GBR_MAX_PRIMES (primes = -1)."""
    from paper_1103_4697_gb300.api import resultant_info

    rng = random.Random(71)
    f, g = _rand_rows(rng, 127, 1, 3), _rand_rows(rng, 127, 1, 3)
    i = resultant_info(f, g)
    assert (i["m"], i["n"]) == (127, 127) and 0 < i["deg_bound"] <= 254
    d = resultant_info(f, None, disc=True)
    assert (d["m"], d["n"]) == (127, 126)
    with pytest.raises(N.GbrError) as e:
        resultant_info(_rand_rows(rng, 128, 1, 3), g)
    assert e.value.status == N.ELIMIT

    big = (1 << 511) - 1                                  # the widest 8-word two's-complement magnitude
    f8, g8 = _rand_rows(rng, 56, 1, big), _rand_rows(rng, 56, 1, big)
    i8 = resultant_info(f8, g8)
    assert 1321 < i8["primes"] <= 2048 and i8["limbs"] > 1280
    assert i8["deg_bound"] == 112
    f9 = [list(r) for r in f8]
    f9[0][0] = 1 << 511                                   # 512 bits and a sign bit: 9 words
    with pytest.raises(N.GbrError) as e:
        resultant_info(f9, g8)
    assert e.value.status == N.EINVAL
    i64 = resultant_info(_rand_rows(rng, 64, 1, big), _rand_rows(rng, 64, 1, big))
    assert i64["primes"] == -1                            # more than the table's GBR_MAX_PRIMES primes


def _is_prime(v):
    if v < 2 or v % 2 == 0:
        return v == 2
    d = 3
    while d * d <= v:
        if v % d == 0:
            return False
        d += 2
    return True


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """include/gbres.h compiles as C99 (-Wall -Wextra -pedantic -Werror) and a C
    program linked against libgbres.so gets the host-only answers: the table's
    two largest primes below 2^32 / 3 that are 1 mod 2^14, prime counts (-1 beyond the table), the
    plan of res_y(x^2 + y^2 - 25, y + x - 1) and of its projection resultant,
    GBR_EINVAL for var = 2, and a status string."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "c_abi_example")
    libdir = os.path.dirname(N.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    "-o", exe, os.path.join(ROOT, "tests", "native", "c_abi_example.c"), "-L", libdir, "-lgbres",
                    "-Wl,-rpath," + libdir], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    top = (2 ** 32 - 1) // 3 // (1 << 14) * (1 << 14) + 1
    want_p = [v for v in range(top, top - 400 * (1 << 14), -(1 << 14)) if _is_prime(v)][:2]
    assert out[0] == "num_primes 2048"
    assert out[1] == f"primes 0 {want_p[0]} {want_p[1]}"
    assert out[2] == "primes_for_bits 4 -1"            # 3 primes give about 91 bits, 4 about 121
    # m = 2, n = 1; D = min(n deg_x f + m deg_x g, Bezout 2 * 1) = min(4, 2) = 2; one prime
    assert out[3] == "info 0 2 1 2 1"
    assert out[4] == "disc 0 2 1 2"                    # f_y = 2y: D = min(1 * 2 + 2 * 0, 2 * 1) = 2
    assert out[5] == f"bad_var {N.EINVAL}"
    assert out[6] == "strerror " + lib.gbr_strerror(N.ELIMIT).decode()


def test_struct_layouts_match_the_header(tmp_path):
    """Every structure of include/gbres.h has the same size, field names, field
    order and field offsets in the binding's ctypes classes as a C compiler
    gives it (tests/native/struct_layout.c)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "struct_layout")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    "-o", exe, os.path.join(ROOT, "tests", "native", "struct_layout.c")], check=True,
                   capture_output=True, text=True)
    lines = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, lines):
        name, size, *fields = line.split()
        cls = getattr(N, name)
        assert C.sizeof(cls) == int(size), name
        c_fields = [(f.split(":")[0], int(f.split(":")[1])) for f in fields]
        assert [f[0] for f in cls._fields_] == [f for f, _ in c_fields], name
        for f, off in c_fields:
            assert getattr(cls, f).offset == off, (name, f)
        seen += 1
    assert seen == 10


_CTYPE_OF = {
    "int": {C.c_int}, "int32_t": {C.c_int32, C.c_int}, "int64_t": {C.c_int64}, "uint64_t": {C.c_uint64},
    "size_t": {C.c_size_t}, "double": {C.c_double}, "void": {None},
}


def _pointer_ok(ctype, c_decl):
    """A C pointer parameter may be passed as c_void_p, as POINTER(...) of a matching
    type, or (const char *) as c_char_p."""
    if ctype in (C.c_void_p, C.c_char_p):
        return True
    return hasattr(ctype, "_type_") and isinstance(ctype._type_, type)


def test_binding_signatures_match_the_header():
    """Each prototype of include/gbres.h and the binding's ctypes declaration agree
    on the return type, the number of arguments and each argument's kind (integer
    width, floating point, or pointer)."""
    text = open(os.path.join(ROOT, "include", "gbres.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"((?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**)\s*(gbr_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text)
    names = set()
    for ret, name, params in protos:
        names.add(name)
        res, args = N.SIGNATURES[name]
        ret = ret.strip()
        if "*" in ret:
            assert res in (C.c_char_p, C.c_void_p), name
        else:
            assert res in _CTYPE_OF[ret.replace("const", "").strip()], (name, ret)
        params = [p.strip() for p in params.split(",")] if params.strip() not in ("", "void") else []
        assert len(params) == len(args), name
        for p, a in zip(params, args):
            if "*" in p:
                assert _pointer_ok(a, p), (name, p)
            else:
                base = re.sub(r"\b(const|unsigned)\b", "", p).split()[0]
                assert a in _CTYPE_OF[base], (name, p, a)
    assert names == set(N.SIGNATURES)


def test_binding_constants_match_the_header():
    """Status codes, options and job kinds of the binding equal the header's
    #define values (GBR_X in include/gbres.h is X in the binding)."""
    text = open(os.path.join(ROOT, "include", "gbres.h")).read()
    defs = dict(re.findall(r"#define\s+GBR_([A-Z0-9_]+)\s+(-?\d+)", text))
    checked = 0
    for name, value in defs.items():
        if name.startswith("MAX_") or name.startswith("NOALLOC_"):
            continue                                      # limits: not mirrored by the binding
        assert getattr(N, name) == int(value), name
        checked += 1
    assert checked == 10 + 9 + 3                          # statuses, options, job kinds


def test_host_bound_at_least_the_exact_bound(lib):
    """gbr_resultant_info's bound (double precision, host) against the oracle's exact
    enclosure of the same Hadamard bound on the GPU test's shapes: the primes it plans
    satisfy M > 2B + 1 for the exact B, and its log2 B is not below the exact value by
    more than its double-precision rounding."""
    from fractions import Fraction

    import test_gpu_bound as TB
    from oracle.bound import log2_floor_half_pred, resultant_bound_log2
    from paper_1103_4697_gb300.api import primes, resultant_info

    jobs = [(f, g, False) for f, g in TB.bound_pairs()[::2]] + [(f, None, True) for f in TB.disc_polys()]
    table = primes(400)
    checked = 0
    for f, g, disc in jobs:
        ex = resultant_bound_log2(f, O.deriv_y(f) if disc else g)
        info = resultant_info(f, g, disc=disc)
        if ex is None:
            continue
        hi = ex[1]
        assert Fraction(info["log2_bound"]) >= hi - Fraction(1, 10 ** 9) * (1 + abs(hi)), (info, float(hi))
        M = 1
        for p in table[:info["primes"]]:
            M *= p
        assert log2_floor_half_pred(M) > hi, (info, float(hi))
        checked += 1
    assert checked >= 80
