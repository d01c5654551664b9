"""Debye polynomials u_k(t) of the uniform large-order expansion (CPU only).

Pins: the first polynomials as printed in DLMF 10.41.10, the recurrence of
paper Eqs. "u0"/"uk" checked symbolically, the committed header equal to a
fresh generation, and the truncation error of U_K against the oracle falling
like v^-(K+1) (it is an asymptotic expansion in 1/v).
"""
import os
import sys
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_08729_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_debye  # noqa: E402


def test_first_polynomials_match_dlmf():
    ps = gen_debye.debye_polys()
    assert ps[1] == {1: F(1, 8), 3: F(-5, 24)}
    assert ps[2] == {2: F(81, 1152), 4: F(-462, 1152), 6: F(385, 1152)}
    assert ps[3] == {3: F(30375, 414720), 5: F(-369603, 414720), 7: F(765765, 414720), 9: F(-425425, 414720)}
    assert ps[4] == {4: F(4465125, 39813120), 6: F(-94121676, 39813120), 8: F(349922430, 39813120),
                     10: F(-446185740, 39813120), 12: F(185910725, 39813120)}


def test_recurrence_residual_is_zero():
    sympy = pytest.importorskip("sympy")
    t, s = sympy.symbols("t s")
    ps = gen_debye.debye_polys()

    def poly(d, var):
        return sum(sympy.Rational(c.numerator, c.denominator) * var ** p for p, c in d.items())

    for k in range(13):
        uk, uk1 = poly(ps[k], t), poly(ps[k + 1], t)
        rhs = (t ** 2 - t ** 4) / 2 * sympy.diff(uk, t) + sympy.Rational(1, 8) * sympy.integrate(
            (1 - 5 * s ** 2) * poly(ps[k], s), (s, 0, t))
        assert sympy.expand(uk1 - rhs) == 0


def test_large_coefficients_and_values_at_one():
    """u_13 has coefficients near 1.1e12 while u_13(1) is only -6.4e-3."""
    cs = gen_debye.p_coeffs(13)
    assert 1.0e12 < max(abs(float(c)) for c in cs) < 1.2e12
    assert abs(float(sum(cs)) + 6.403e-3) < 1e-5


def test_header_is_current(tmp_path):
    out = tmp_path / "debye_uk.h"
    text = gen_debye.render_header(gen_debye.debye_polys())
    with open(os.path.join(CSRC, "debye_uk.h")) as f:
        assert f.read() == text


def test_uniform_expansion_truncation_order():
    """|U_K - log I_v| shrinks by about 2^(K+1) each time v doubles (x = v)."""
    mp = pytest.importorskip("mpmath")
    import oracle
    mp.mp.dps = 40
    K = 4
    pcs = {k: [mp.mpf(c.numerator) / c.denominator for c in gen_debye.p_coeffs(k)] for k in range(1, K + 1)}

    def u_expr(v, x):
        v, x = mp.mpf(v), mp.mpf(x)
        xp = x / v
        r = mp.sqrt(1 + xp * xp)
        t = 1 / r
        eta = r + mp.log(xp / (1 + r))
        S = 1 + sum(t ** k * mp.polyval(pcs[k][::-1], t * t) / v ** k for k in range(1, K + 1))
        return -mp.log(2 * mp.pi * v) / 2 + v * eta - mp.log(1 + xp * xp) / 4 + mp.log(S)

    errs = []
    for v in (8.0, 16.0, 32.0, 64.0):
        hi, lo = oracle.log_i([v], [v], want_lo=True)
        errs.append(abs(u_expr(v, v) - (mp.mpf(hi[0]) + mp.mpf(lo[0]))))
    ratios = [float(errs[i] / errs[i + 1]) for i in range(3)]
    for r in ratios:
        assert 2 ** (K + 1) * 0.6 < r < 2 ** (K + 1) * 1.6, ratios
