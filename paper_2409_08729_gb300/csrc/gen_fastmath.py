"""Generate the tables of lb_fastmath.cuh (needs mpmath).

Table-driven exp and log in the manner of P. T. P. Tang, "Table-driven
implementation of the exponential function in IEEE floating-point arithmetic"
(ACM TOMS 15(2), 1989) and "Table-driven implementation of the logarithm
function in IEEE floating-point arithmetic" (ACM TOMS 16(4), 1990):

  exp: 2^(j/512), j = 0..511, as a double-double (hi + lo).
  log: for m = 1 + (j + 1/2)/128 (the midpoints of the 128 mantissa intervals
       of [1, 2)), c_j = 1/m rounded to 24 bits, and -log(c_j) as a
       double-double; for m >= sqrt(2) the entry is -log(c_j) - log(2) so that
       the reduction is centred on 1; the intervals touching 1 use c = 1 and
       c = 1/2 with zero entries (log of arguments near 1 stays accurate
       relative to its size).
"""
import os
import struct
import sys

import mpmath as mp

mp.mp.dps = 60


def dd(x):
    hi = float(x)
    lo = float(x - mp.mpf(hi))
    return hi, lo


def f24(x):
    """Round to a float (24-bit significand), returned as a Python float."""
    return struct.unpack("f", struct.pack("f", float(x)))[0]


def main():
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "fastmath_tables.h")
    lines = ["// Generated by gen_fastmath.py -- do not edit.", "#pragma once", ""]
    ehi, elo = [], []
    for j in range(512):
        h, l = dd(mp.mpf(2) ** (mp.mpf(j) / 512))
        ehi.append(h)
        elo.append(l)
    ch, lh, ll = [], [], []
    sqrt2 = mp.sqrt(2)
    for j in range(128):
        m = 1 + (mp.mpf(j) + mp.mpf(0.5)) / 128
        c = f24(1 / m)
        # The two intervals next to 1 ([1, 1 + 1/128) and, after the centring,
        # [1 - 1/256, 1)) use c = 1 and c = 1/2 exactly, so the table entry is
        # 0 and log(1 + r) is formed from r = z - 1 alone: no cancellation
        # between table and polynomial for arguments near 1.
        if j == 0:
            c = 1.0
        if j == 127:
            c = 0.5
        val = -mp.log(mp.mpf(c))
        if 1 + mp.mpf(j) / 128 >= sqrt2:
            val -= mp.log(2)
        h, l = dd(val)
        ch.append(c)
        lh.append(h)
        ll.append(l)
    # first index whose interval starts at or above sqrt(2)
    jsplit = next(j for j in range(128) if 1 + mp.mpf(j) / 128 >= sqrt2)

    def arr(name, vals):
        body = ",\n  ".join(", ".join(repr(v) for v in vals[i:i + 4]) for i in range(0, len(vals), 4))
        return "static __device__ const double %s[%d] = {\n  %s};\n" % (name, len(vals), body)

    lines.append("#define LB_FM_LOG_JSPLIT %d" % jsplit)
    lines.append(arr("lb_fm_exp_hi", ehi))
    lines.append(arr("lb_fm_exp_lo", elo))
    lines.append(arr("lb_fm_log_c", ch))
    lines.append(arr("lb_fm_log_hi", lh))
    lines.append(arr("lb_fm_log_lo", ll))
    # reduction constants for exp: 512/ln2, ln2/512 split so that k * hi is exact for |k| < 2^20
    inv = float(512 / mp.log(2))
    l = mp.log(2) / 512
    hi_bits = struct.unpack("<Q", struct.pack("<d", float(l)))[0] & ~((1 << 20) - 1)   # keep 33 bits
    lhi = struct.unpack("<d", struct.pack("<Q", hi_bits))[0]
    llo = float(l - mp.mpf(lhi))
    lines.append("#define LB_FM_INV_L %r" % inv)
    lines.append("#define LB_FM_L_HI %r" % lhi)
    lines.append("#define LB_FM_L_LO %r" % llo)
    # ln 2 split so that e * hi is exact for |e| < 2^11 (hi keeps 42 bits)
    ln2 = mp.log(2)
    b = struct.unpack("<Q", struct.pack("<d", float(ln2)))[0] & ~((1 << 11) - 1)
    ln2h = struct.unpack("<d", struct.pack("<Q", b))[0]
    ln2l = float(ln2 - mp.mpf(ln2h))
    lines.append("#define LB_FM_LN2_HI %r" % ln2h)
    lines.append("#define LB_FM_LN2_LO %r" % ln2l)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
