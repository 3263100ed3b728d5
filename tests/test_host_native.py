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
    out = subprocess.run([exe, "1500", "2000"], check=True, capture_output=True, text=True).stdout.split("\n")
    n = int(out[0])
    i, bad = 1, []
    for case in range(n):
        a, b, q, r, g1, g2 = (_int(out[i + k]) for k in range(6))
        i += 6
        if (q, r) != divmod(a, b) or g1 != math.gcd(a, b) or g2 != math.gcd(a, b):
            bad.append(case)
    assert n == 3500 and not bad, bad[:10]


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


def _kron(rows, D):
    z = {}
    for j, r in enumerate(rows):
        for i, c in enumerate(r):
            if c:
                z[i + j * D] = c
    n = max(z) + 1 if z else 0
    return [z.get(k, 0) for k in range(n)]


def _unkron(coefs, D, off):
    rows = {}
    for k, c in enumerate(coefs):
        if c:
            i, j = (k + off) % D, (k + off) // D
            rows.setdefault(j, {})[i] = c
    if not rows:
        return []
    out = []
    for j in range(max(rows) + 1):
        r = rows.get(j, {})
        out.append(tuple(r.get(i, 0) for i in range(max(r) + 1)) if r else ())
    return out


def _shift_rows(rows, s):
    """rows (row j = Z[x] coefficients of y^j) -> the same polynomial at y + s."""
    if not rows:
        return []
    dy, w = len(rows) - 1, max(len(r) for r in rows)
    c = [list(r) + [0] * (w - len(r)) for r in rows]
    for i in range(w):
        for k in range(dy):
            for j in range(dy - 1, k - 1, -1):
                c[j][i] += s * c[j + 1][i]
    out = [tuple(r) for r in c]
    out = [tuple(_trim_t(r)) for r in out]
    while out and not out[-1]:
        out.pop()
    return out


def _trim_t(r):
    r = list(r)
    while r and r[-1] == 0:
        r.pop()
    return r


def test_kronecker_shift_choice(tmp_path):
    """The bivariate gcd's candidate choice on the CPU: for random pairs (and pairs
    whose images share a power of z, or a common zero at (1, 1), that is not a common
    factor), the Kronecker images' gcd and cofactors come from the oracle; with the
    candidate the harness picks, D + 1 while none passes and, after four values of D,
    the inputs shifted by y -> y + s (as the library does), the map-back shifted back
    equals the oracle's gcd_zxy and exact quotients."""
    import random

    import oracle as O

    exe = _build(tmp_path, "kron_harness.cpp")
    rng = random.Random(61)

    def rand2(dy, dx, amp):
        f = [[rng.randint(-amp, amp) for _ in range(dx + 1)] for _ in range(dy + 1)]
        f[dy][rng.randint(0, dx)] = rng.choice([1, -1, 2])
        return f

    def mul2(a, b):
        out = [[0] * (max(len(r) for r in a) + max(len(r) for r in b) - 1) for _ in range(len(a) + len(b) - 1)]
        for j1, r1 in enumerate(a):
            for i1, c1 in enumerate(r1):
                for j2, r2 in enumerate(b):
                    for i2, c2 in enumerate(r2):
                        out[j1 + j2][i1 + i2] += c1 * c2
        return out

    pairs = [([[0, 1], [1]], [[0, 1], [-1]]), ([[0, 0], [0, 1]], [[0, 0, 1]])]
    for _ in range(150):
        h = rand2(rng.randint(0, 2), rng.randint(0, 2), 3)
        u, v = rand2(rng.randint(0, 2), rng.randint(0, 2), 4), rand2(rng.randint(0, 2), rng.randint(0, 2), 4)
        if rng.random() < 0.3:                      # no constant terms: images share powers of z
            u, v = mul2(u, [[0, 1], [rng.choice([1, -1, 2])]]), mul2(v, [[0, 1], [rng.choice([1, -1, 3])]])
        pairs.append((mul2(h, u), mul2(h, v)))
    n = len(pairs)
    D0 = [max(max(len(r) for r in a), max(len(r) for r in b)) for a, b in pairs]
    D, ys, tries = list(D0), [0] * n, [0] * n
    pend, done, shifted = list(range(n)), 0, 0
    for _ in range(40):
        if not pend:
            break
        lines, data = [str(len(pend))], []
        for k in pend:
            a, b = pairs[k]
            if ys[k]:
                a, b = _shift_rows(a, ys[k]), _shift_rows(b, ys[k])
            za, zb = _kron(a, D[k]), _kron(b, D[k])
            G = list(O.gcd_z(za, zb))
            Ga = list(O.zx_divexact(O.zx_trim(za), tuple(G))) if G else []
            Gb = list(O.zx_divexact(O.zx_trim(zb), tuple(G))) if G else []
            data.append((G, Ga, Gb))
            lines.append(str(D[k]))
            for p in (G, Ga, Gb):
                lines.append(" ".join([str(len(p) - 1)] + [str((c > 0) - (c < 0)) for c in p]))
        res = subprocess.run([exe], input="\n".join(lines) + "\n", check=True, capture_output=True, text=True)
        cand = [int(t) for t in res.stdout.split()]
        retry = []
        for k, t, (G, Ga, Gb) in zip(pend, cand, data):
            if t < 0:
                D[k] += 1
                tries[k] += 1
                if tries[k] == 4:
                    ys[k] += 1
                    assert ys[k] <= 3, k
                    D[k], tries[k] = D0[k], 0
                retry.append(k)
                continue
            a, b = pairs[k]
            H = O.gcd_zxy(a, b)
            assert _shift_rows(_unkron(G, D[k], -t), -ys[k]) == H, k
            assert _shift_rows(_unkron(Ga, D[k], t), -ys[k]) == O.divexact_zxy(a, H), k
            assert _shift_rows(_unkron(Gb, D[k], t), -ys[k]) == O.divexact_zxy(b, H), k
            done += 1
            shifted += ys[k] > 0
        pend = retry
    assert not pend and done == n
    assert shifted >= 1                     # the (1, 1) case took the shifted path


def _limbs(v):
    m, out = abs(v), []
    while m:
        out.append(m & 0xFFFFFFFF)
        m >>= 32
    return out


def _taylor(rows, s):
    """rows[j][i] of f(x, y) -> rows of f(x, y + s) by the binomial theorem."""
    dy, w = len(rows) - 1, len(rows[0])
    out = [[0] * w for _ in range(dy + 1)]
    for j in range(dy + 1):
        for k in range(j + 1):
            c = math.comb(j, k) * s ** (j - k)
            for i in range(w):
                out[k][i] += c * rows[j][i]
    return out


def test_kronecker_host_helpers(tmp_path):
    """The bivariate gcd's int64 shift y -> y + s (exact, or refused on int64
    overflow), the big-integer shift back, the partial derivatives of an int64 curve
    and the two's-complement packing of big cofactors, against Python integers
    (binomial expansions, plain products, two's-complement decoding)."""
    import random

    exe = _build(tmp_path, "kron_ops_harness.cpp")
    rng = random.Random(62)
    I64 = (-(1 << 63), (1 << 63) - 1)
    cmds, checks = [], []

    def flat(rows):
        return [c for r in rows for c in r]

    def unflat(v, dx, dy):
        return [v[j * (dx + 1):(j + 1) * (dx + 1)] for j in range(dy + 1)]

    for _ in range(300):                                     # S: y -> y + s in int64
        dx, dy, s = rng.randint(0, 4), rng.randint(0, 6), rng.randint(1, 3)
        big = rng.random() < 0.3
        amp = (1 << rng.randint(50, 62)) if big else 1000
        rows = [[rng.randint(-amp, amp) for _ in range(dx + 1)] for _ in range(dy + 1)]
        cmds.append(" ".join(map(str, ["S", dx, dy, s] + flat(rows))))
        checks.append(("S", rows, s, dx, dy))
    for _ in range(200):                                     # U: y -> y - s in big integers
        dx, dy, s = rng.randint(0, 3), rng.randint(0, 6), rng.randint(1, 3)
        rows = [[rng.choice([0, rng.randint(-(1 << 300), 1 << 300)]) for _ in range(dx + 1)] for _ in range(dy + 1)]
        words = ["U", dx, dy, s]
        for c in flat(rows):
            l = _limbs(c)
            words += [(c > 0) - (c < 0), len(l)] + l
        cmds.append(" ".join(map(str, words)))
        checks.append(("U", rows, s, dx, dy))
    for _ in range(200):                                     # D: derivatives in x and y
        dx, dy, wx = rng.randint(0, 5), rng.randint(0, 5), rng.randint(0, 1)
        amp = (1 << 61) if rng.random() < 0.3 else 1 << 20
        rows = [[rng.randint(-amp, amp) for _ in range(dx + 1)] for _ in range(dy + 1)]
        cmds.append(" ".join(map(str, ["D", wx, dx, dy] + flat(rows))))
        checks.append(("D", rows, wx, dx, dy))
    for _ in range(200):                                     # W: two's-complement words
        dx, dy, L = rng.randint(0, 3), rng.randint(-1, 3), rng.randint(1, 17)
        nco = (dx + 1) * (dy + 1) if dy >= 0 else 0
        vals = [rng.choice([0, rng.randint(-(1 << (32 * L)) + 1, (1 << (32 * L)) - 1)]) for _ in range(nco)]
        words = ["W", dx, dy, L]
        for c in vals:
            l = _limbs(c) + [0] * L
            words += [(c > 0) - (c < 0)] + l[:L]
        cmds.append(" ".join(map(str, words)))
        checks.append(("W", vals, L, dx, dy))

    res = subprocess.run([exe], input="\n".join(cmds) + "\n", check=True, capture_output=True, text=True)
    lines = res.stdout.splitlines()
    assert len(lines) == len(checks)
    seen = {"OVF": 0, "LIMIT": 0}
    for line, (op, a, b, dx, dy) in zip(lines, checks):
        t = line.split()
        if op == "S":
            want = flat(_taylor(a, b))
            fits = all(I64[0] <= v <= I64[1] for v in want)
            small = all(abs(c) <= 1000 for c in flat(a))
            if t[0] == "OVF":
                assert not small, line                       # small inputs never overflow
                seen["OVF"] += 1
            else:
                assert [int(v) for v in t[1:]] == want
            if not fits:
                assert t[0] == "OVF"
        elif op == "U":
            want, got, k = flat(_taylor(a, -b)), [], 0
            while k < len(t):
                sg, nl = int(t[k]), int(t[k + 1])
                got.append(sg * sum(int(v) << (32 * q) for q, v in enumerate(t[k + 2:k + 2 + nl])))
                k += 2 + nl
            assert got == want
            assert flat(_taylor(unflat(got, dx, dy), b)) == flat(a)        # the shift back inverts the shift
        elif op == "D":
            if b:   # d/dx
                ox, oy = max(dx - 1, 0), dy
                want = [[(i + 1) * a[j][i + 1] if i + 1 <= dx else 0 for i in range(ox + 1)] for j in range(oy + 1)]
            else:
                ox, oy = dx, max(dy - 1, 0)
                want = [[(j + 1) * a[j + 1][i] if j + 1 <= dy else 0 for i in range(ox + 1)] for j in range(oy + 1)]
            fits = all(I64[0] <= v <= I64[1] for v in flat(want))
            if fits:
                assert t[:3] == ["OK", str(ox), str(oy)] and [int(v) for v in t[3:]] == flat(want), line
            else:
                assert t == ["OVF"]
                seen["OVF"] += 1
        else:
            L, W = b, (32 * b + 1 + 63) // 64
            if dy < 0:                                   # zero: one coefficient 0, whatever L
                assert t == ["OK", "0", "0", "1", "0"]
                continue
            if W > 8:
                assert t == ["LIMIT"]
                seen["LIMIT"] += 1
                continue
            assert t[0] == "OK"
            assert t[1:4] == [str(dx), str(dy), str(W)]
            w = [int(v) for v in t[4:]]
            got = []
            for c in range(len(a)):
                u = sum(w[c * W + q] << (64 * q) for q in range(W))
                got.append(u - (1 << (64 * W)) if u >> (64 * W - 1) else u)
            assert got == a
    assert seen["OVF"] > 0 and seen["LIMIT"] > 0


def _table_primes(k):
    """The k largest primes below 2^32 / 3 that are 1 mod 2^14 (the library's table)."""
    step = 1 << 14
    out, v = [], (2 ** 32 - 1) // 3 // step * step + 1
    while len(out) < k:
        if all(v % d for d in range(3, int(v ** 0.5) + 1, 2)):
            out.append(v)
        v -= step
    return out


def test_elimination_routines_match_sylvester_determinants(tmp_path):
    """The evaluation kernels' per-(prime, point) resultant, run on the CPU through
    its host path: res_formal (every case of the formal-degree recursion) and the
    register form res_chain<N> for N = 2..32 in all three shapes, against the
    oracle's integer resultant reduced mod p - the Sylvester determinant with the
    formal degrees where a leading coefficient vanishes, the subresultant sequence
    over Z otherwise.  Cases: random residues, zero leading coefficients (one or
    both), polynomials even in y (remainder sequences that are not normal), a
    planted common root mod p, constants and small residues."""
    import random

    from oracle.resultant import det_bareiss, res_univariate, sylvester
    from oracle.zpoly import ZZ

    exe = _build(tmp_path, "elim_harness.cpp")
    rng = random.Random(63)
    primes = _table_primes(3)

    def poly_mul_mod(a, b, p):
        out = [0] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            for j, y in enumerate(b):
                out[i + j] = (out[i + j] + x * y) % p
        return out

    cases = []
    for N in range(2, 33):
        for m, n in ((N, N), (N, N - 1), (N - 1, N)):
            for kind in ("rand", "rand", "even", "root"):
                cases.append((m, n, kind))
    for _ in range(500):
        cases.append((rng.randint(0, 9), rng.randint(0, 9), rng.choice(["rand", "lc0", "lc00", "even", "root", "small"])))
    lines, want = [], []
    for m, n, kind in cases:
        p = rng.choice(primes)
        pick = (lambda: rng.choice([0, 1, 2, p - 1])) if kind == "small" else (lambda: rng.randrange(p))
        f = [pick() for _ in range(m + 1)]
        g = [pick() for _ in range(n + 1)]
        if kind == "even":                               # only even powers of y
            f = [c if k % 2 == 0 else 0 for k, c in enumerate(f)]
            g = [c if k % 2 == 0 else 0 for k, c in enumerate(g)]
        if kind == "root" and m >= 1 and n >= 1:         # a common root r mod p: the resultant is 0
            r = rng.randrange(p)
            f = poly_mul_mod([(p - r) % p, 1], [rng.randrange(p) for _ in range(m)], p)
            g = poly_mul_mod([(p - r) % p, 1], [rng.randrange(p) for _ in range(n)], p)
        if kind == "lc0":
            f[-1] = 0
        if kind == "lc00":
            f[-1] = 0
            g[-1] = 0
        if f[-1] and g[-1]:
            v = res_univariate(list(f), list(g), ZZ) if m and n else (g[0] ** m if not n else f[0] ** n)
        else:
            v = det_bareiss(sylvester(list(f), list(g), ZZ), ZZ)
        want.append(v % p)
        lines.append(" ".join(map(str, [p, m, n] + f + g)))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", check=True, capture_output=True, text=True).stdout
    got = [tuple(int(t) for t in l.split()) for l in out.splitlines()]
    assert len(got) == len(cases)
    reg_ok = reg_total = 0
    for (m, n, kind), w, (formal, ok, chain) in zip(cases, want, got):
        assert formal == w, (m, n, kind)
        N = max(m, n)
        if 2 <= N <= 32 and {m, n} <= {N, N - 1}:
            reg_total += 1
            if ok:
                reg_ok += 1
                assert chain == w, (m, n, kind)
            else:
                # the register form declines only where a leading coefficient
                # vanishes or the sequence is not normal (the kernel's redo pass)
                assert kind in ("even", "lc0", "lc00", "small", "root") or w == 0, (m, n, kind)
    assert reg_ok > reg_total // 2


def test_montgomery_arithmetic_at_the_range_ends(tmp_path):
    """The kernels' Montgomery arithmetic (host paths of gbr_modarith.cuh) for the
    table's largest primes: products, the fused two- and three-product forms with
    residues up to p (the sum stays below p 2^32 only because p < 2^32 / 3),
    conversions, powers, inverses and multi-word two's-complement reduction
    (including -2^511 and all-ones words), against Python's modular integers."""
    import random

    exe = _build(tmp_path, "modarith_harness.cpp")
    rng = random.Random(64)
    lines, want = [], []
    for p in _table_primes(2) + [(1 << 30) + 3]:           # the largest table primes and one near 2^30
        Ri = pow(1 << 32, -1, p)
        ends = [0, 1, p - 1, p - 2, p // 2]

        def r(upto=p - 1):
            return rng.choice(ends + [upto]) if rng.random() < 0.5 else rng.randint(0, upto)

        for _ in range(150):
            a, b = r(), r()
            lines.append(f"mul {p} {a} {b}"); want.append(a * b * Ri % p)
            a, x, b, y = r(), r(), r(), r()
            lines.append(f"mulsub {p} {a} {x} {b} {y}"); want.append((a * x - b * y) * Ri % p)
            a, x, b, y = r(p), r(p), r(p), r(p)
            lines.append(f"fma2 {p} {a} {x} {b} {y}"); want.append((a * x + b * y) * Ri % p)
            a, x, b, y, c, z = r(p), r(p), r(p), r(p), r(p), r(p)
            lines.append(f"fma3 {p} {a} {x} {b} {y} {c} {z}"); want.append((a * x + b * y + c * z) * Ri % p)
            v = rng.choice([0, 1, (1 << 32) - 1, rng.getrandbits(32)])
            lines.append(f"to {p} {v}"); want.append(v * (1 << 32) % p)
            lines.append(f"from {p} {r()}"); want.append(None)
            xx, e = r(), rng.randint(0, 70)
            lines.append(f"pow {p} {xx} {e}"); want.append(pow(xx, e, p))
            if xx:
                lines.append(f"inv {p} {xx}"); want.append(pow(xx, -1, p))
            W = rng.randint(1, 8)
            v = rng.choice([-(1 << (64 * W - 1)), (1 << (64 * W - 1)) - 1, -1, 0, rng.getrandbits(64 * W - 1),
                            -rng.getrandbits(64 * W - 1)])
            u = v % (1 << (64 * W))
            words = [(u >> (64 * i)) & ((1 << 64) - 1) for i in range(W)]
            lines.append(f"words {p} {W} " + " ".join(map(str, words))); want.append(v % p)
    out = subprocess.run([exe], input="\n".join(lines) + "\n", check=True, capture_output=True, text=True).stdout.split()
    assert len(out) == len(lines)
    for line, w, g in zip(lines, want, out):
        g = int(g)
        assert 0 <= g < int(line.split()[1]), line
        if line.startswith("from"):
            p, xv = (int(t) for t in line.split()[1:3])
            assert g * (1 << 32) % p == xv % p, line        # from inverts the Montgomery map
        else:
            assert g == w, line


def test_routing_helpers(tmp_path):
    """reg_shape sends exactly the shapes (N, N), (N, N-1), (N-1, N) with 2 <= N <= 32
    to the register form; the symmetric points run 0, +1, -1, +2, -2, ... (the
    unit grid otherwise); the even and odd interpolation matrices use the points
    j^2 and (j + 1)^2; rows4 pads m + 1 rows to a multiple of 4; a root-of-unity set
    has the next power of two (at least 64) points, and the point-set choice follows
    the measured crossover on its shapes; shared point counts only raise a count to a
    larger one of the same batch, in runs that stay within 1/16 (at least 4 points) of
    their smallest count, from 512 points on never cross a power of two (the root-of-unity
    set) and
    stop growing at a full tile of 128 pairs."""
    nvcc = shutil.which("nvcc")
    cuda = os.environ.get("CUDA_HOME") or (os.path.dirname(os.path.dirname(nvcc)) if nvcc else "")
    inc = os.path.join(cuda, "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    exe = _build(tmp_path, "routing_harness.cpp", ["-I", inc])
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines()
    seen = {"reg": 0, "pt": 0, "rows4": 0, "rootn": 0, "roots": 0, "quad": 0, "share": 0}
    shared = {}
    # expected point-set choice per crossover shape: degree-20 and -24 batches and full
    # tiles stay on integer points; small batches, long rows and point counts above the
    # cached contraction's range take roots of unity; without the contraction, always roots
    want_roots = {(401, 4096): 0, (577, 1024): 0, (257, 1024): 0, (8193, 8): 1, (4097, 8): 1, (1025, 8): 1,
                  (401, 8): 1, (16001, 4000): 1}
    for line in out:
        t = line.split()
        seen[t[0]] += 1
        v = [int(x) for x in t[1:]]
        if t[0] == "rootn":
            P, N = v
            assert N >= max(64, P) and N & (N - 1) == 0 and (N == 64 or N // 2 < P), line
            continue
        if t[0] == "roots":
            P, tf, tg, m, n, share, auto, nogemm = v
            assert auto == want_roots[(P, share)] and nogemm == 1, line
            continue
        if t[0] == "share":
            b, P, pairs, to = v
            shared.setdefault(b, []).append((P, pairs, to))
            continue
        if t[0] == "quad":
            # the points 0 and i^k a (a = 1..h) cover the P coefficients; R_t holds the
            # coefficients 4 r + t < P
            P, h, pe, pairs, r0, r1, r2, r3 = v
            assert 4 * h + 1 >= P > 4 * (h - 1) + 1 or (P == 1 and h == 0), line
            assert pe == 4 * h + 4 and pairs == 2 * h + 1, line   # three pads after the point 0
            assert [r0, r1, r2, r3] == [len(range(t, P, 4)) for t in range(4)], line
            assert r0 <= h + 1 and max(r1, r2, r3) <= h, line
            continue
        if t[0] == "reg":
            m, n, N = v
            top = max(m, n)
            want = top if 2 <= top <= 32 and min(m, n) >= top - 1 else 0
            assert N == want, line
        elif t[0] == "pt":
            j, grid, sym, vsym, even, odd = v
            s = 0 if j == 0 else ((j + 1) // 2 if j % 2 else -(j // 2))
            assert (grid, sym, vsym, even, odd) == (j, s, s, j * j, (j + 1) ** 2), line
        else:
            m, r = v
            assert r % 4 == 0 and m + 1 <= r < m + 5, line
    assert seen["reg"] == 41 * 41 and seen["pt"] == 64 and seen["rows4"] == 131 and seen["roots"] == 8
    assert seen["quad"] == 64
    for b, rows in shared.items():
        counts = [P for P, _, _ in rows]
        for P, _, to in rows:
            assert to >= P and to in counts
        runs = {}
        for P, pairs, to in rows:
            runs.setdefault(to, []).append((P, pairs))
        tos = sorted(runs)
        for k, to in enumerate(tos):
            members = sorted(runs[to])
            lo = members[0][0]
            assert members[-1][0] == to and to <= lo + max(4, lo // 16), (b, members)
            rootn = lambda P: max(64, 1 << (P - 1).bit_length())
            assert lo < 512 or rootn(to) == rootn(lo), (b, members)
            # consecutive counts of the batch; every count but the last joined while the
            # run held fewer than 128 pairs
            i0 = counts.index(lo)
            assert [P for P, _ in members] == counts[i0:i0 + len(members)]
            assert sum(p for _, p in members[:-1]) < 128, (b, members)
            # a run ends at a full tile, at the batch's end, or before a count too far away
            if k + 1 < len(tos):
                nxt = sorted(runs[tos[k + 1]])[0][0]
                assert (sum(p for _, p in members) >= 128 or nxt > lo + max(4, lo // 16)
                        or (lo >= 512 and rootn(nxt) != rootn(lo))), (b, members, nxt)
    assert shared[0] == [(61, 6, 65), (65, 4, 65), (67, 2, 71), (71, 4, 71), (73, 4, 73)]
    assert shared[1] == [(401, 4096, 401)]
    assert [to for _, _, to in shared[2]] == [33, 37, 37]
    assert [to for _, _, to in shared[6]] == [1024, 1024, 1050, 1050]
    assert seen["rootn"] > 1100


def test_host_constant_tables(tmp_path):
    """The host-built tables every Chinese remaindering and Newton interpolation
    launch reads: the table primes (the largest primes below 2^32 / 3 that are
    1 mod 2^14, in descending order) with pinv = -p^-1 mod 2^32, r1 = 2^32 mod p, r2 = 2^64 mod p;
    the Garner prefix table ((p_0 ... p_{i-1})^-1 and p_j mod p_i, Montgomery form);
    the inverse table (1/t mod p_i, Montgomery form); the warp Chinese remaindering
    table (Garner rows (-p_0 ... p_{j-1}) R mod p_i, limbs of p_0 ... p_{i-1}),
    against their definitions."""
    if not os.path.exists(N.LIB_PATH):
        from paper_1103_4697_gb300.build import build
        build()
    nvcc = shutil.which("nvcc")
    cuda = os.environ.get("CUDA_HOME") or (os.path.dirname(os.path.dirname(nvcc)) if nvcc else "")
    inc = os.path.join(cuda, "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    libdir = os.path.dirname(N.LIB_PATH)
    exe = _build(tmp_path, "tables_harness.cpp", ["-I", inc, "-L", libdir, "-lgbres", "-Wl,-rpath," + libdir])
    K, T = 40, 300
    out = subprocess.run([exe, str(K), str(T)], check=True, capture_output=True, text=True).stdout.split("\n")
    assert int(out[0]) == 2048
    mods = [tuple(int(v) for v in out[1 + i].split()) for i in range(K)]
    ps = [m[0] for m in mods]
    assert ps == _table_primes(K)
    R = 1 << 32
    for p, pinv, r1, r2 in mods:
        assert (p * pinv) % R == R - 1 and r1 == R % p and r2 == (R * R) % p
    g = [int(v) for v in out[1 + K].split()]
    assert len(g) == K + K * (K - 1) // 2
    for i, p in enumerate(ps):
        prod = 1
        for j in range(i):
            assert g[K + i * (i - 1) // 2 + j] == ps[j] % p * R % p
            prod = prod * ps[j] % p
        assert g[i] == pow(prod, -1, p) * R % p
    inv = [int(v) for v in out[2 + K].split()]
    assert len(inv) == K * T
    for i, p in enumerate(ps):
        assert inv[i * T] == 0
        for t in range(1, T):
            assert inv[i * T + t] == pow(t, -1, p) * R % p
    LW = int(out[3 + K])
    assert LW == (31 * K + 31) // 32
    w = [int(v) for v in out[4 + K].split()]
    assert len(w) == K * (K - 1) // 2 + K * LW
    for i, p in enumerate(ps):
        for j in range(i):
            prod = 1
            for t in range(j):
                prod *= ps[t]
            assert w[i * (i - 1) // 2 + j] == (-prod) % p * R % p
    prod = 1
    for i in range(K):
        row = w[K * (K - 1) // 2 + i * LW:K * (K - 1) // 2 + (i + 1) * LW]
        assert sum(v << (32 * l) for l, v in enumerate(row)) == prod
        prod *= ps[i]


def test_device_prime_table_bytes(tmp_path):
    """The device prime table as the host builds it: (R^3, R^4) mod p per prime, and
    the Chinese-remaindering tables of the first 64 primes that the fast path
    reads - Garner row i at crt_gd_off(i) holds (-prod_{l<j} p_l) R mod p_i for
    j < i and zeros in its padding; limb l of prod_{j<i} p_j for i <= 64; the first
    non-zero column of each limb row, rounded down to a multiple of 4."""
    if not os.path.exists(N.LIB_PATH):
        from paper_1103_4697_gb300.build import build
        build()
    nvcc = shutil.which("nvcc")
    cuda = os.environ.get("CUDA_HOME") or (os.path.dirname(os.path.dirname(nvcc)) if nvcc else "")
    inc = os.path.join(cuda, "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    libdir = os.path.dirname(N.LIB_PATH)
    exe = _build(tmp_path, "prime_table_harness.cpp", ["-I", inc, "-L", libdir, "-lgbres", "-Wl,-rpath," + libdir])
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    NP, size = (int(v) for v in out[0].split())
    K, ROW, L = 64, 68, 62
    R = 1 << 32
    ps = []
    for i in range(K):
        p, r3, r4 = (int(v) for v in out[1 + i].split())
        assert r3 == pow(R, 3, p) and r4 == pow(R, 4, p)
        ps.append(p)
    assert ps == _table_primes(K)

    def gd_off(i):
        if i <= 0:
            return 0
        q, r = (i - 1) // 4, (i - 1) % 4
        return 8 * q * (q + 1) + 4 * r * (q + 1)

    gd = [int(v) for v in out[1 + K].split()]
    assert len(gd) == gd_off(K)
    expect = [0] * gd_off(K)
    for i in range(1, K):
        C = 1
        for j in range(i):
            expect[gd_off(i) + j] = (-C) % ps[i] * R % ps[i]
            C = C * ps[j] % ps[i]
    assert gd == expect
    T = [[int(v) for v in out[2 + K + l].split()] for l in range(L)]
    prod = 1
    for i in range(K + 1):
        for l in range(L):
            assert T[l][i] == (prod >> (32 * l)) & (R - 1), (l, i)
        if i < K:
            prod *= ps[i]
    I0 = [int(v) for v in out[2 + K + L].split()]
    for l in range(L):
        first = next((i for i in range(K + 1) if T[l][i]), K + 1)    # a row of zeros: past the end
        assert I0[l] == first & ~3
    # root-of-unity tables: per prime T1[j] = w^j R, T2[j] = w^(128 j) R (mod p) with w of
    # order exactly 2^14
    roots = [[int(v) for v in out[3 + K + L + t].split()] for t in range(K + 2)]
    for t, row in enumerate(roots):
        p = ps[t] if t < K else int(row[0])
        vals = row[1:] if t >= K else row
        assert len(vals) == 256
        w = vals[1] * pow(R, -1, p) % p
        assert pow(w, 1 << 14, p) == 1 and pow(w, 1 << 13, p) == p - 1
        for j in range(128):
            assert vals[j] == pow(w, j, p) * R % p and vals[128 + j] == pow(w, 128 * j, p) * R % p
        # the quartic point set reads i = w^(2^12) (R i) straight from T2[32]: i^2 = -1
        iota = vals[128 + 32] * pow(R, -1, p) % p
        assert iota * iota % p == p - 1 and vals[0] == R % p
    assert size == NP * (16 + 8 + 256 * 4) + (gd_off(K) + L * ROW + L) * 4


def test_no_int8_tensor_mma_on_sm103a(tmp_path):
    """The interpolation contraction uses bf16 digits because GB300 has no int8 MMA:
    the assembler refuses tcgen05.mma kind::i8 for sm_103a (and accepts it for sm_100a),
    while kind::f16 (the library's) and kind::f8f6f4 assemble for sm_103a."""
    nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    src = tmp_path / "mma_kinds.cu"

    def kernel(kind):
        return ('__global__ void k_%s(unsigned d, unsigned long long a, unsigned long long b, unsigned i, '
                'unsigned c) { asm volatile("{\\n\\t.reg .pred p;\\n\\tsetp.ne.u32 p, %%4, 0;\\n\\t'
                'tcgen05.mma.cta_group::1.kind::%s [%%0], %%1, %%2, %%3, p;\\n\\t}" :: "r"(d), "l"(a), "l"(b), '
                '"r"(i), "r"(c)); }\n' % (kind, kind))

    def assemble(arch, kind):
        src.write_text(kernel(kind))
        r = subprocess.run([nvcc, "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", str(src), "-o",
                            str(tmp_path / "k.o")], capture_output=True, text=True)
        return r.returncode, r.stdout + r.stderr

    rc, out = assemble("103a", "i8")
    assert rc != 0 and "kind::i8" in out and "not supported" in out, out
    assert assemble("100a", "i8")[0] == 0
    assert assemble("103a", "f16")[0] == 0
    assert assemble("103a", "f8f6f4")[0] == 0
