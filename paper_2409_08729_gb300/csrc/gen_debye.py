"""Generate the Debye polynomials u_k(t), k = 0..13, as exact rationals and
write them as a CUDA header of double-precision Horner coefficients.

u_0(t) = 1 and
u_{k+1}(t) = (t^2 - t^4)/2 * u_k'(t) + 1/8 * int_0^t (1 - 5 s^2) u_k(s) ds
(paper Sec. 3.1, Eqs. "u0" and "uk"; DLMF 10.41.9).  u_k has the form
t^k * P_k(t^2) with deg P_k = k, so the header stores the k+1 coefficients of
P_k in ascending powers of p = t^2.  The paper prints none of u_7..u_13; they
are generated here from the recurrence with Python's exact Fractions.

Usage: python gen_debye.py [output.h]   (default: debye_uk.h beside this file)
"""
import os
import sys
from fractions import Fraction

import numpy as np

KMAX = 13


def debye_polys(kmax=KMAX):
    """Return [u_0, ..., u_kmax], each a dict power -> Fraction."""
    polys = [{0: Fraction(1)}]
    for _ in range(kmax):
        u = polys[-1]
        nxt = {}
        # (t^2 - t^4)/2 * u'(t)
        for p, c in u.items():
            if p == 0:
                continue
            d = c * p                    # coefficient of t^(p-1)
            nxt[p + 1] = nxt.get(p + 1, 0) + d / 2
            nxt[p + 3] = nxt.get(p + 3, 0) - d / 2
        # 1/8 * int_0^t (1 - 5 s^2) u(s) ds
        for p, c in u.items():
            nxt[p + 1] = nxt.get(p + 1, 0) + c / (8 * (p + 1))
            nxt[p + 3] = nxt.get(p + 3, 0) - 5 * c / (8 * (p + 3))
        polys.append({p: c for p, c in nxt.items() if c != 0})
    return polys


def p_coeffs(k, polys=None):
    """Coefficients of P_k in ascending powers of p = t^2, where u_k = t^k P_k(t^2)."""
    polys = polys or debye_polys()
    u = polys[k]
    out = [Fraction(0)] * (k + 1)
    for p, c in u.items():
        assert (p - k) % 2 == 0 and 0 <= (p - k) // 2 <= k, (k, p)
        out[(p - k) // 2] = c
    return out


def q_coeffs(k, polys=None):
    """Coefficients of Q_k(p) = k P_k(p) + 2 p P_k'(p), ascending in p = t^2.

    With u_k(t) = t^k P_k(t^2), d/dt u_k(t) = t^(k-1) Q_k(t^2); the
    x-derivative of the uniform expansion needs these."""
    pc = p_coeffs(k, polys)
    return [k * c + 2 * j * c for j, c in enumerate(pc)]


def _horner(cs, fn_name):
    expr = repr(float(cs[-1]))
    for j in range(len(cs) - 2, -1, -1):
        expr = "fma(%s, p, %s)" % (expr, repr(float(cs[j])))
    lines = ["template <typename T> __host__ __device__ __forceinline__ T %s(T p) {" % fn_name,
             "  return %s;" % expr.replace("fma(", "lb_fma<T>("), "}", ""]
    return lines


def f32_split(c):
    """c (a Fraction) as a pair of floats hi + lo: hi = c rounded to single
    precision, lo = the remainder rounded to single precision (exact
    Fraction arithmetic, one rounding each)."""
    import struct

    def to_f32(q):
        # nearest float to the rational q: round through a double, then fix
        # the rare double-rounding case by comparing the two neighbours
        f = struct.unpack("f", struct.pack("f", float(q)))[0]
        best, err = f, abs(Fraction(f) - q)
        for g in (np.nextafter(np.float32(f), np.float32(np.inf)), np.nextafter(np.float32(f), np.float32(-np.inf))):
            e = abs(Fraction(float(g)) - q)
            if e < err:
                best, err = float(g), e
        return best

    hi = to_f32(c)
    lo = to_f32(c - Fraction(hi))
    return hi, lo


def _f32_lit(f):
    """A float as an exact C hexadecimal literal with the f suffix."""
    if f == 0.0:
        return "0.0f"
    return float(f).hex() + "f"


def render_header(polys):
    lines = [
        "// Generated by gen_debye.py -- do not edit.",
        "// Debye polynomials u_k(t) = t^k P_k(t^2), k = 1..13, from the recurrence",
        "// u_{k+1} = (t^2 - t^4)/2 u_k' + 1/8 int_0^t (1 - 5 s^2) u_k ds, u_0 = 1",
        "// (paper Sec. 3.1, Eqs. \"u0\" and \"uk\"), exact rationals rounded to double.",
        "#pragma once",
        "",
        "#define LB_DEBYE_KMAX %d" % KMAX,
        "",
    ]
    for k in range(1, KMAX + 1):
        cs = p_coeffs(k, polys)
        lines.append("// P_%d(p), coefficients ascending: %s" % (k, ", ".join(str(c) for c in cs)))
        lines += _horner(cs, "lb_debye_P%d" % k)
    lines.append("// The same coefficients as a table: lb_debye_c[k][i] = coefficient of t^(k+2i)")
    lines.append("// in u_k(t) (k = 0..13, i = 0..k; zero beyond), for sums formed per block.")
    rows = []
    for k in range(KMAX + 1):
        cs = p_coeffs(k, polys) if k > 0 else [Fraction(1)]
        rows.append("  {" + ", ".join(repr(float(c)) for c in cs + [Fraction(0)] * (KMAX + 1 - len(cs))) + "}")
    lines.append("static __device__ const double lb_debye_c[%d][%d] = {\n%s};" % (KMAX + 1, KMAX + 1, ",\n".join(rows)))
    lines.append("")
    lines.append("// Q_k(p) = k P_k(p) + 2 p P_k'(p): d/dt u_k(t) = t^(k-1) Q_k(t^2)")
    lines.append("")
    for k in range(1, KMAX + 1):
        lines += _horner(q_coeffs(k, polys), "lb_debye_Q%d" % k)
    lines.append("// P_k(p) in double-float (lb_df.cuh), k = 2..13: each coefficient as the")
    lines.append("// pair hi + lo of floats nearest to it (exact hexadecimal literals), in one")
    lines.append("// table: the k + 1 coefficients of P_k, ascending, from lb_debye_df_off[k].")
    offs, rows, o = [0, 0], [], 0
    for k in range(2, KMAX + 1):
        offs.append(o)
        for c in p_coeffs(k, polys):
            hi, lo = f32_split(c)
            rows.append("  {%s, %s}" % (_f32_lit(hi), _f32_lit(lo)))
        o += k + 1
    lines.append("#define LB_DEBYE_DF_N %d" % o)
    lines.append("static __constant__ const int lb_debye_df_off[%d] = {%s};" % (KMAX + 1, ", ".join(map(str, offs))))
    lines.append("static __constant__ const float lb_debye_df[%d][2] = {\n%s};" % (o, ",\n".join(rows)))
    lines.append("// Q_k(p) in double-float, k = 2..13, the same layout (Q_k has the degree")
    lines.append("// of P_k): the k + 1 coefficients of Q_k, ascending, from lb_debye_df_off[k].")
    qrows = []
    for k in range(2, KMAX + 1):
        for c in q_coeffs(k, polys):
            hi, lo = f32_split(c)
            qrows.append("  {%s, %s}" % (_f32_lit(hi), _f32_lit(lo)))
    assert len(qrows) == o
    lines.append("static __constant__ const float lb_debye_qdf[%d][2] = {\n%s};" % (o, ",\n".join(qrows)))
    lines.append("")
    return "\n".join(lines) + "\n"


def main():
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "debye_uk.h")
    text = render_header(debye_polys())
    with open(out, "w") as f:
        f.write(text)


if __name__ == "__main__":
    main()
