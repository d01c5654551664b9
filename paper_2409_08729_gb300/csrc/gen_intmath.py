"""Generate the tables of lb_intmath.cuh (needs mpmath).

Fixed-point exp and log on the integer pipes, after the table-driven methods
of P. T. P. Tang (ACM TOMS 15(2), 1989 and 16(4), 1990), with the arithmetic
in 64- and 128-bit integers instead of doubles:

  exp: T_j = 2^(j/512) in Q62, j = 0..511; ln2/512 in Q116 (128 bits).
  log: C_j = 2^13 / m_j rounded to an integer, m_j = 1 + (j + 1/2)/512 the
       midpoints of the 512 mantissa intervals of [1, 2) (C_0 = 2^13 and
       C_511 = 2^12 exactly, so that arguments next to 1 keep their relative
       accuracy), and -log(C_j / 2^13) in Q116 (128 bits, signed); ln 2 in
       Q116 (the entry for j = 511 is this same constant).
  Horner coefficients of e^r - 1 and log(1 + r) in Q31 (inner steps, done
  with 32-bit multiplies) and Q62.
  Fixed-point forms for sums of exponentials of logarithms (the K-integral
       nodes, ix_log_q53 and ix_exp_q58_fx): -log(C_j / 2^13) in Q62; ln 2
       as A 2^-30 + B 2^-62 + C 2^-94 (A, B, C integers below 2^32); ln2/512
       as (H + M 2^-32) 2^-64; the log's coefficients 1/3..1/5 in Q30.
  rcp and rsqrt reuse the log's C_j (m C_j / 2^13 = 1 + r): 1/m =
       (C_j / 2^13) / (1 + r), m^-1/2 = sqrt(C_j / 2^13) (1 + r)^-1/2, with
       sqrt(C_j / 2^13) in Q63 and the binomial coefficients of
       (1 + r)^-1/2 (dyadic rationals) in Q30 and Q62.
"""
import os
import sys

import mpmath as mp

mp.mp.dps = 80


def q(x, bits):
    return int(mp.nint(mp.mpf(x) * mp.mpf(2) ** bits))


def split128(v):
    """Signed 128-bit integer -> (hi as int64, lo as uint64)."""
    v &= (1 << 128) - 1
    hi, lo = v >> 64, v & ((1 << 64) - 1)
    if hi >= 1 << 63:
        hi -= 1 << 64
    return hi, lo


def main():
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                            "intmath_tables.h")
    L = ["// Generated by gen_intmath.py -- do not edit.", "#pragma once", "", "#include <stdint.h>", ""]

    def arr(ctype, name, vals, fmt):
        body = ",\n  ".join(", ".join(fmt(v) for v in vals[i:i + 4]) for i in range(0, len(vals), 4))
        return "LB_IX_TABLE %s %s[%d] = {\n  %s};\n" % (ctype, name, len(vals), body)

    u64 = lambda v: "0x%016xull" % v
    exp_t = [q(mp.mpf(2) ** (mp.mpf(j) / 512), 62) for j in range(512)]
    assert all(v < 1 << 63 for v in exp_t)
    L.append(arr("uint64_t", "lb_ix_exp_t", exp_t, u64))
    ln2 = q(mp.log(2), 116)
    c, th, tl = [], [], []
    for j in range(512):
        if j == 0:
            cj = 1 << 13
        elif j == 511:
            cj = 1 << 12
        else:
            cj = int(mp.nint(mp.mpf(2) ** 13 / (1 + (mp.mpf(j) + mp.mpf(0.5)) / 512)))
        c.append(cj)
        t = 0 if j == 0 else (ln2 if j == 511 else q(-mp.log(mp.mpf(cj) / 2 ** 13), 116))
        hi, lo = split128(t)
        th.append(hi)
        tl.append(lo)
    L.append(arr("uint16_t", "lb_ix_log_c", c, lambda v: "%d" % v))
    L.append(arr("int64_t", "lb_ix_log_thi", th, lambda v: "%dll" % v))
    L.append(arr("uint64_t", "lb_ix_log_tlo", tl, u64))
    t62 = [0 if j == 0 else q(-mp.log(mp.mpf(cj) / 2 ** 13), 62) for j, cj in enumerate(c)]
    assert all(abs(v) < 1 << 62 for v in t62) and t62[511] == q(mp.log(2), 62)
    L.append(arr("int64_t", "lb_ix_log_t62", t62, lambda v: "%dll" % v))
    hi, lo = split128(q(mp.log(2) / 512, 116))
    L.append("#define LB_IX_L512_HI %dull" % hi)
    L.append("#define LB_IX_L512_LO 0x%016xull" % lo)
    hi, lo = split128(ln2)
    L.append("#define LB_IX_LN2_HI %dull" % hi)
    L.append("#define LB_IX_LN2_LO 0x%016xull" % lo)
    l96 = q(mp.log(2) / 512, 96)
    L.append("#define LB_IX_L512_H %dull" % (l96 >> 32))
    L.append("#define LB_IX_L512_M %dull" % (l96 & 0xffffffff))
    # e^r - 1 = r (1 + r (1/2 + r (1/6 + r (1/24 + r/120)))): the inner three
    # coefficients in Q31 (32-bit steps), the outer two in Q62
    for k in (3, 4, 5):
        L.append("#define LB_IX_E%d %d" % (k, q(1 / mp.factorial(k), 31)))
    for k in (1, 2):
        L.append("#define LB_IX_E%d %dll" % (k, q(1 / mp.factorial(k), 62)))
    # log(1 + r) = r (1 - r (1/2 - r (1/3 - r (1/4 - r (1/5 - r/6))))): 1/4..1/6
    # in Q31, 1/1..1/3 in Q62
    for k in (4, 5, 6):
        L.append("#define LB_IX_L%d %d" % (k, q(mp.mpf(1) / k, 31)))
    for k in (1, 2, 3):
        L.append("#define LB_IX_L%d %dll" % (k, q(mp.mpf(1) / k, 62)))
    # the Q53 log (ix_log_q53) takes r in Q64 and stops at r^5: 1/3, 1/4 and
    # 1/5 in Q30, -log(C_j / 2^13) in Q62, ln 2 as A 2^-30 + B 2^-62 + C 2^-94
    for k in (3, 4, 5):
        L.append("#define LB_IX_LQ%d %d" % (k, q(mp.mpf(1) / k, 30)))
    l94 = q(mp.log(2), 94)
    assert l94 >> 64 < 1 << 30
    L.append("#define LB_IX_LN2Q_A %dll" % (l94 >> 64))
    L.append("#define LB_IX_LN2Q_B %dll" % ((l94 >> 32) & 0xffffffff))
    L.append("#define LB_IX_LN2Q_C %dll" % (l94 & 0xffffffff))
    # rsqrt: sqrt(C_j / 2^13) in Q63 (at most 2^63, for j = 0)
    rsq = [q(mp.sqrt(mp.mpf(cj) / 2 ** 13), 63) for cj in c]
    assert all(v <= 1 << 63 for v in rsq)
    L.append(arr("uint64_t", "lb_ix_rsq_t", rsq, u64))
    # (1 + r)^-1/2 = 1 - r (1/2 - r (3/8 - r (5/16 - r (35/128 - r (63/256 - r 231/1024))))):
    # the coefficients binom(2k, k) / 4^k; 3..6 in Q30, 1..2 in Q62 (all exact)
    for k in range(1, 7):
        ck = mp.binomial(2 * k, k) / mp.mpf(4) ** k
        if k >= 3:
            L.append("#define LB_IX_R%d %d" % (k, q(ck, 30)))
        else:
            L.append("#define LB_IX_R%d %dll" % (k, q(ck, 62)))
    L.append("#define LB_IX_RSQRT_HALF 0x%016xull" % q(1 / mp.sqrt(2), 64))
    with open(out, "w") as f:
        f.write("\n".join(L) + "\n")


if __name__ == "__main__":
    main()
