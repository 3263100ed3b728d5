"""CPU oracle for the exact bivariate resultant and the univariate integer gcd.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
big-integer restatement of what the GPU library computes.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library itself never does, and shares no code, table or constant with
it (the oracle has no primes, no residues, no Chinese remaindering).

What it computes (Berberich, Emeliyanenko, Kobel, Sagraloff, "Arrangement
Computation for Planar Algebraic Curves"):

* Section 2.1 (Projection Phase) uses R = res(f, f_y, y) in Z[x]; Section 3
  (Arrangement Computation) uses R_CD = res(f, g, y) and notes that R_CD vanishes
  where f(alpha, y) and g(alpha, y) share a root *or both leading coefficients
  vanish*, i.e. the resultant is the Sylvester determinant taken with the
  degrees of f and g as polynomials in y over Z[x].  Section 4 ("Symbolic
  Speedups") says resultants and gcds are the only symbolic operations and are
  computed by the modular method of Brown and Collins; the oracle does not follow
  that method, it evaluates the definition.
* Section 2 (Algorithm) and 2.1 use gcds of univariate integer polynomials
  (content removal, square-free factorisation).

Functions
---------
``res_bareiss``   determinant of the Sylvester matrix over Z[x], fraction-free
                  Bareiss elimination (the definition).
``res_leibniz``   the same determinant by permutation expansion (tiny inputs).
``res_subres``    subresultant polynomial remainder sequence over Z[x][y].
``res_evalz``     exact evaluation at integer points x = a, integer resultant per
                  point, exact Newton interpolation over Z (no primes).
``res_at``        exact R(a) for one integer a (Sylvester determinant at x = a).
``disc_res``      res_y(f, df/dy).
``gcd_z``         primitive polynomial remainder sequence over Z.
``sqf_yun``       square-free factorisation R = u prod r_i^i (Section 2.1) by Yun's
                  algorithm over Z with primitive gcds.
``gcd_zxy``       gcd in Z[x][y] by the primitive remainder sequence over Z[x];
                  ``content_y`` (content removal, Section 2), ``teissier_q``
                  (Q = res(f_x/h, f_y/h, y), h = gcd(f_x, f_y), Section 2.1).

Every function is pinned by ``tests/test_oracle.py`` against closed forms
(planted roots), invariants (symmetry, multiplicativity, planted common factor),
brute force on tiny inputs and, where available, sympy.
"""

from .zpoly import (ZZ, ZX, zx_add, zx_sub, zx_mul, zx_neg, zx_trim, zx_eval, zx_divexact,
                    zx_deg, content, primitive_part)
from .resultant import (sylvester, det_bareiss, res_bareiss, res_leibniz, res_subres, res_evalz, res_at_prs,
                        res_at, disc_res, deriv_y, ydeg, xdeg, res_univariate, degree_bound)
from .gcd import gcd_z, divides_z
from .sqf import sqf_yun
from . import bigcd
from .bigcd import content_y, divexact_zxy, gcd_zxy, teissier_parts, teissier_q

__all__ = [
    "ZZ", "ZX", "zx_add", "zx_sub", "zx_mul", "zx_neg", "zx_trim", "zx_eval", "zx_divexact",
    "zx_deg", "content", "primitive_part", "sylvester", "det_bareiss", "res_bareiss", "res_leibniz",
    "res_subres", "res_evalz", "res_at", "res_at_prs", "disc_res", "deriv_y", "ydeg", "xdeg", "res_univariate",
    "degree_bound", "gcd_z", "divides_z", "sqf_yun", "bigcd", "content_y", "divexact_zxy", "gcd_zxy",
    "teissier_parts", "teissier_q",
]
