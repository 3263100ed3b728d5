"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake (a dropped term, a wrong sign, index or divisor, a
transposed operand) in a temporary copy of ``oracle/`` and runs the pins of
``tests/test_oracle.py`` against that copy in a child process: at least one
pin must fail (pytest exit status 1).  The unchanged copy must pass (status 0),
so a failure comes from the planted mistake and not from the copying.  A
mistake that makes the oracle loop forever counts as caught when a pin runs
past its time limit (pytest-timeout, 30 s per pin; every pin takes well under
a second).  The repository's own ``oracle/`` is never modified.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

pytest.importorskip("pytest_timeout")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file under oracle/, text as written, text with the mistake)
MUTATIONS = [
    # Sylvester matrix (Section 2.1 definition of res_y as det Syl_y)
    ("sylvester_f_row_reversed", "resultant.py", "M[r][r + t] = F[m - t]", "M[r][r + t] = F[t]"),
    ("sylvester_g_row_shifted", "resultant.py", "M[n + r][r + t] = G[n - t]", "M[n + r][(r + t + 1) % N] = G[n - t]"),
    # Bareiss elimination
    ("bareiss_swap_keeps_sign", "resultant.py", "sign = -sign", "sign = sign"),
    ("bareiss_divisor_not_updated", "resultant.py", "        prev = akk\n", "        prev = prev\n"),
    ("bareiss_transposed_product", "resultant.py", "ring.mul(aik, A[k][j])", "ring.mul(A[k][j], A[j][k])"),
    # subresultant remainder sequence
    ("subres_h_update_dropped", "resultant.py",
     "h = ring.divexact(_pow(g, delta, ring), _pow(h, delta - 1, ring))", "h = g"),
    ("subres_sign_rule", "resultant.py", "if da % 2 and db % 2:", "if da % 2 or db % 2:"),
    ("subres_swap_sign_dropped", "resultant.py", "        if (da * db) % 2:\n            s = -s\n",
     "        if (da * db) % 2:\n            pass\n"),
    ("subres_divisor_power", "resultant.py", "div = ring.mul(g, _pow(h, delta, ring))", "div = ring.mul(g, _pow(h, delta - 1, ring))"),
    ("prem_extra_power", "resultant.py", "for k in range(len(A) - 1, db - 1, -1):", "for k in range(len(A), db - 1, -1):"),
    ("subres_final_power", "resultant.py",
     "v = ring.divexact(_pow(B[0], da, ring), _pow(h, da - 1, ring)) if da >= 1 else ring.one",
     "v = _pow(B[0], da, ring)"),
    # degree bound, evaluation and interpolation
    ("degree_bound_short", "resultant.py", "return max(0, n * dxf + m * dxg)", "return max(0, n * dxf + m * dxg - 1)"),
    ("interp_node_off_by_one", "resultant.py", "zx_mul(poly, (-(a0 + j), 1))", "zx_mul(poly, (-(a0 + j + 1), 1))"),
    ("res_at_ignores_point", "resultant.py", "Fa = [zx_eval(c, a) for c in F]", "Fa = [zx_eval(c, a + 1) for c in F]"),
    ("deriv_y_factor", "resultant.py", "[(j + 1) * c for c in F[j + 1]]", "[j * c for c in F[j + 1]]"),
    # Z[x] arithmetic
    ("zx_mul_overwrites", "zpoly.py", "out[i + j] += c * d", "out[i + j] = c * d"),
    ("primitive_part_sign", "zpoly.py", "    if a[-1] < 0:\n        g = -g", "    if a[-1] > 0:\n        g = -g"),
    ("zx_sub_adds", "zpoly.py", "return zx_add(a, zx_neg(b))", "return zx_add(a, b)"),
    # gcd in Z[x]
    ("gcd_content_dropped", "gcd.py", "return tuple(c * x for x in g)", "return tuple(g)"),
    ("gcd_prem_unscaled", "gcd.py", "r = [lb * x for x in r]", "r = [x for x in r]"),
    ("gcd_zero_argument_sign", "gcd.py", "return tuple(-c for c in p) if p[-1] < 0 else p", "return p"),
    # Yun's square-free factorisation
    ("yun_derivative_term_dropped", "sqf.py", "d = zx_sub(zx_divexact(d, ri), _deriv(c))", "d = zx_divexact(d, ri)"),
    ("yun_initial_d", "sqf.py", "d = zx_sub(zx_divexact(b, g), _deriv(c))", "d = zx_divexact(b, g)"),
    ("yun_unit_sign", "sqf.py", "u = content(r) * (1 if r[-1] > 0 else -1)", "u = content(r)"),
    ("yun_derivative_factor", "sqf.py", "return zx_trim(i * a[i] for i in range(1, len(a)))",
     "return zx_trim(a[i] for i in range(1, len(a)))"),
    # bivariate gcd, content and the Teissier Q
    ("bigcd_content_gcd_dropped", "bigcd.py", "return _normalise([zx_mul(c, row) for row in H])", "return _normalise(H)"),
    ("bigcd_normalise_wrong_coefficient", "bigcd.py", "if rows and rows[-1][-1] < 0:", "if rows and rows[-1][0] < 0:"),
    ("content_y_last_row_only", "bigcd.py", "g = gcd_z(g, row)", "g = gcd_z((), row)"),
    ("divexact_zxy_sign", "bigcd.py", "A[k + t] = zx_sub(A[k + t], zx_mul(q, B[t]))", "A[k + t] = zx_add(A[k + t], zx_mul(q, B[t]))"),
    ("teissier_no_division_by_h", "bigcd.py", "return h, divexact_zxy(fx, h), divexact_zxy(fy, h)", "return h, fx, fy"),
    ("teissier_deriv_x_factor", "bigcd.py", "tuple(i * row[i] for i in range(1, len(row)))",
     "tuple(row[i] for i in range(1, len(row)))"),
    ("teissier_deriv_y_factor", "bigcd.py", "tuple((j + 1) * c for c in F[j + 1])", "tuple(j * c for c in F[j + 1])"),
    ("teissier_operands_swapped", "bigcd.py",
     "return res_subres([list(r) or [0] for r in fxs], [list(r) or [0] for r in fys])",
     "return res_subres([list(r) or [0] for r in fys], [list(r) or [0] for r in fxs])"),
    ("teissier_zero_not_trimmed", "bigcd.py", "    if not fxs or not fys:\n        return ()\n",
     "    if not fxs or not fys:\n        return (0,)\n"),
    ("pp_y_no_division", "bigcd.py", "return [zx_divexact(r, c) if r else () for r in F] if c else []", "return F"),
    ("content_y_skips_first_row", "bigcd.py", "    for row in as_zxy(f):\n        g = gcd_z(g, row)",
     "    for row in as_zxy(f)[1:]:\n        g = gcd_z(g, row)"),
    # more of the resultant's definition and evaluation
    ("evalz_window_ignores_g", "resultant.py", "zx_eval(lf, a) * zx_eval(lg, a) == 0", "zx_eval(lf, a) == 0"),
    ("bareiss_pivot_search_skips_a_row", "resultant.py", "for i in range(k + 1, n) if not ring.is_zero(A[i][k])",
     "for i in range(k + 2, n) if not ring.is_zero(A[i][k])"),
    ("res_at_operands_swapped", "resultant.py", "return det_bareiss(sylvester(Fa, Ga, ZZ), ZZ)",
     "return det_bareiss(sylvester(Ga, Fa, ZZ), ZZ)"),
    ("subres_constant_power", "resultant.py",
     "        v = _pow(B[0], da, ring)\n        return v if s > 0 else ring.neg(v)\n    g = ring.one",
     "        v = _pow(B[0], max(da - 1, 0), ring)\n        return v if s > 0 else ring.neg(v)\n    g = ring.one"),
    ("leibniz_sign_dropped", "resultant.py",
     "total = ring.add(total, term) if _perm_sign(p) > 0 else ring.sub(total, term)", "total = ring.add(total, term)"),
    ("degree_bound_transposed", "resultant.py", "return max(0, n * dxf + m * dxg)", "return max(0, m * dxf + n * dxg)"),
    ("deriv_y_drops_top_row", "resultant.py", "for j in range(len(F) - 1)]", "for j in range(len(F) - 2)]"),
    ("zx_eval_sign", "zpoly.py", "v = v * x + c", "v = v * x - c"),
    ("primitive_part_keeps_content", "zpoly.py", "    g = content(a)\n    if a[-1] < 0:", "    g = 1\n    if a[-1] < 0:"),
    ("gcd_content_of_one_argument", "gcd.py", "c = math.gcd(content(p), content(q))", "c = content(p)"),
    ("yun_quotient_not_divided", "sqf.py", "        c = zx_divexact(c, ri)\n", "        c = c[1:] or c\n"),
    # the coefficient bound (Hadamard's inequality on the scaled Sylvester matrix)
    ("bound_autocorr_factor_two", "bound.py", "g += 2 * abs(", "g += abs("),
    # the summed forms: |C_k| after the sum over the entries, lambda^(2 deg), the factor 2
    ("summed_abs_per_entry", "bound.py", "            I[k][t % 4] += a << (t // 4)\n",
     "            I[k][t % 4] += abs(a) << (t // 4)\n"),
    ("summed_lambda_exponent", "bound.py", "        t = d * q8\n", "        t = 2 * d * q8\n"),
    ("summed_factor_two", "bound.py", "        slo, shi = slo + 2 * lo, shi + 2 * hi\n",
     "        slo, shi = slo + lo, shi + hi\n"),
    ("bound_autocorr_no_abs", "bound.py", "g += 2 * abs(sum(h[a] * h[a + k] for a in range(L - k)))",
     "g += 2 * sum(h[a] * h[a + k] for a in range(L - k))"),
    ("bound_lambda_power_dropped", "bound.py", "lam = Fraction(m * n * q, 4)", "lam = Fraction(m * n * q, 8)"),
    ("bound_rows_counts_swapped", "bound.py", "for s, count in ((sf, n), (sg, m)):", "for s, count in ((sf, m), (sg, n)):"),
    ("bound_column_index", "bound.py", "                x = sf[m - (c - r)]\n", "                x = sf[min(m, c - r)]\n"),
    ("bound_sqrt2_low", "bound.py", "    hi = a + b * _S2_HI\n", "    hi = a + b\n"),
    ("bound_log2_round_down", "bound.py", "return val + Fraction(2, 1 << _T) if up else val", "return val"),
]


def _tree(base, name, mutation):
    """A directory with a copy of oracle/ (one mistake planted), the oracle's pins,
    their fixtures and a link to the input generators."""
    d = os.path.join(base, name)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(d, "tests"))
    for f in ("conftest.py", "test_oracle.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), os.path.join(d, "pytest.ini"))
    os.symlink(os.path.join(ROOT, "paper_1103_4697_gb300"), os.path.join(d, "paper_1103_4697_gb300"))
    if mutation is not None:
        fname, old, new = mutation
        path = os.path.join(d, "oracle", fname)
        src = open(path).read()
        assert src.count(old) == 1, f"{name}: the text to mutate must occur exactly once in oracle/{fname}"
        open(path, "w").write(src.replace(old, new))
    return d


def _run(d):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTHONPATH", None)
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "--timeout", "30", "tests/test_oracle.py"], cwd=d, env=env, capture_output=True, text=True,
                       timeout=300)
    return p.returncode, p.stdout[-2000:] + p.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("mutants"))
    jobs = {"unchanged": _tree(base, "unchanged", None)}
    for name, fname, old, new in MUTATIONS:
        jobs[name] = _tree(base, name, (fname, old, new))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_run, d) for name, d in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unchanged_copy_passes(outcomes):
    rc, out = outcomes["unchanged"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    assert rc == 1, f"the pins did not catch the planted mistake {name} (pytest status {rc}):\n{out}"
