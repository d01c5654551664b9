"""Generate the quadrature tables of the K-integral evaluator (needs mpmath).

The paper evaluates log K_v(x) for small inputs from Rothwell's integral
(paper Sec. 3.2, Eq. "log Kv integral"):

  K_v(x) = sqrt(pi) e^{-x} / (Gamma(v+1/2) (2x)^v) * int_0^inf F(s) ds,
  F(s) = e^{-s} (s (s + 2x))^{v-1/2},

split at s = 1 into g(u) on [0, 1] (s = u^beta, beta = 2n/(2v+1), n = 8) and
h(u) on [0, 1] (s = 1/u).  The paper integrates both with composite Simpson,
N = 600.  These tables hold Gauss rules for the same two pieces instead:

  g piece: Gauss-Legendre in u on [0, 1], 24, 32 or 64 nodes; for small
           orders and tiny arguments (v < 0.4, x < 1e-3) the g piece is split
           at s1 = 128 x: [0, s1] with the 64-node rule in u (s = s1 u^beta),
           [s1, 1] in y = log s with plain Gauss-Legendre panels placed per
           pair (tables of 16 and 32 nodes on [0, 1]).
  h piece: Gauss-Legendre in y = log s on [0, log 100] (s in [1, 100]),
           32, 40 or 48 nodes, for orders v <= 5;
           Gauss-Laguerre in t = s - 1, 32 nodes, for orders v > 5.
  one-slot rules (2 <= v <= 16.5, and 0.9 <= v < 2 for x >= 0.8): the
           split moved from s = 1 to s0, so that the branch point s = 0 of
           (s (s + 2x))^(v-1/2) lies s0 away from the Gauss-Laguerre nodes
           of [s0, inf) (t = s - s0); [0, s0] with s = s0 u^beta and
           Gauss-Legendre in u.  s0 = 8 with 22 + 10 nodes (2 <= v < 7),
           s0 = 3 with 12 + 20 (7 <= v <= 16.5); s0 = 10 with 24 + 8 and
           n = 6 (beta = 12/(2v+1), 0.9 <= v < 2, x >= 0.8).

Writes kquad_tables.h beside this file.  Nodes and weights are computed in
40-digit arithmetic and rounded to double.  The log terms that the values'
fixed-point node sums use (c_j and y_j of the tables the one-slot, packed
and fixed rules take, log 8 and log 3) are also written in Q53 (int64,
round(value 2^53)), rounded from the 40-digit values.
"""
import os
import sys

import mpmath as mp

mp.mp.dps = 40
SMAX = 100


def gauss_legendre01(N):
    xs, ws = [], []
    for k in range(1, N + 1):
        x0 = mp.cos(mp.pi * (k - mp.mpf(0.25)) / (N + mp.mpf(0.5)))
        for _ in range(200):
            p0, p1 = mp.mpf(1), x0
            for j in range(2, N + 1):
                p0, p1 = p1, ((2 * j - 1) * x0 * p1 - (j - 1) * p0) / j
            dp = N * (x0 * p1 - p0) / (x0 * x0 - 1)
            dx = p1 / dp
            x0 -= dx
            if abs(dx) < mp.mpf(10) ** (-38):
                break
        xs.append((1 - x0) / 2)
        ws.append(1 / ((1 - x0 * x0) * dp * dp))
    order = sorted(range(N), key=lambda i: xs[i])
    return [xs[i] for i in order], [ws[i] for i in order]


def gauss_laguerre(N):
    A = mp.matrix(N, N)
    for k in range(N):
        A[k, k] = 2 * k + 1
        if k + 1 < N:
            A[k, k + 1] = A[k + 1, k] = k + 1
    E, Q = mp.eigsy(A)
    pairs = sorted((E[i], Q[0, i] ** 2) for i in range(N))
    return [p[0] for p in pairs], [p[1] for p in pairs]


def arr(name, vals):
    """The table as double, plus a float copy named lb_kqf_* for the FP32 path."""
    import struct
    body = ",\n  ".join(", ".join(repr(float(v)) for v in vals[i:i + 4]) for i in range(0, len(vals), 4))
    fl = [struct.unpack("f", struct.pack("f", float(v)))[0] for v in vals]
    bodyf = ",\n  ".join(", ".join(repr(v) + "f" for v in fl[i:i + 4]) for i in range(0, len(fl), 4))
    return ("static __device__ const double %s[%d] = {\n  %s};\n" % (name, len(vals), body)
            + "static __device__ const float %s[%d] = {\n  %s};\n" % (name.replace("lb_kq_", "lb_kqf_"), len(fl), bodyf))


def arrq(name, vals):
    """The table in Q53: round(value 2^53) as int64, named name + "_q"."""
    q = [int(mp.nint(mp.mpf(v) * mp.mpf(2) ** 53)) for v in vals]
    assert all(abs(v) < 1 << 63 for v in q)
    body = ",\n  ".join(", ".join("%dll" % v for v in q[i:i + 4]) for i in range(0, len(q), 4))
    return "static __device__ const long long %s_q[%d] = {\n  %s};\n" % (name, len(q), body)


def main():
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)), "kquad_tables.h")
    parts = ["// Generated by gen_quad.py -- do not edit.",
             "// Gauss rules for the g and h pieces of the K integral (see gen_quad.py).",
             "#pragma once", "", "#define LB_KQ_SMAX %d" % SMAX, ""]
    for N in (12, 22, 24, 32, 64):
        u, w = gauss_legendre01(N)
        parts.append("// g piece, Gauss-Legendre on [0,1], %d nodes: log u_j and log w_j" % N)
        parts.append(arr("lb_kq_g%d_logu" % N, [mp.log(a) for a in u]))
        parts.append(arr("lb_kq_g%d_logw" % N, [mp.log(a) for a in w]))
        parts.append("// log w_j + (n - 1) log u_j with n = 8 (the u^(n-1) factor of g folded in)")
        parts.append(arr("lb_kq_g%d_c" % N, [mp.log(b) + 7 * mp.log(a) for a, b in zip(u, w)]))
        parts.append(arrq("lb_kq_g%d_c" % N, [mp.log(b) + 7 * mp.log(a) for a, b in zip(u, w)]))
        if N == 24:
            parts.append("// the same with n = 6 (the one-slot rule with s0 = 10)")
            parts.append(arr("lb_kq_g24n6_c", [mp.log(b) + 5 * mp.log(a) for a, b in zip(u, w)]))
            parts.append(arrq("lb_kq_g24n6_c", [mp.log(b) + 5 * mp.log(a) for a, b in zip(u, w)]))
    for N in (16, 32):
        t, w = gauss_legendre01(N)
        parts.append("// plain Gauss-Legendre on [0,1], %d nodes: t_j and log w_j (panels placed per pair)" % N)
        parts.append(arr("lb_kq_gl%d_t" % N, t))
        parts.append(arr("lb_kq_gl%d_logw" % N, [mp.log(a) for a in w]))
    Y = mp.log(SMAX)
    for N in (32, 40, 48):
        y, w = gauss_legendre01(N)
        ys = [a * Y for a in y]
        parts.append("// h piece, Gauss-Legendre in y = log s on [0, log %d], %d nodes:" % (SMAX, N))
        parts.append("// s_j, y_j and log(w_j * log(%d)) + y_j - s_j (weight, Jacobian ds = s dy, e^{-s})" % SMAX)
        parts.append(arr("lb_kq_hl%d_s" % N, [mp.exp(a) for a in ys]))
        parts.append(arr("lb_kq_hl%d_y" % N, ys))
        parts.append(arr("lb_kq_hl%d_c" % N, [mp.log(wj * Y) + yj - mp.exp(yj) for wj, yj in zip(w, ys)]))
        parts.append(arrq("lb_kq_hl%d_y" % N, ys))
        parts.append(arrq("lb_kq_hl%d_c" % N, [mp.log(wj * Y) + yj - mp.exp(yj) for wj, yj in zip(w, ys)]))
    t, lam = gauss_laguerre(32)
    parts.append("// h piece, Gauss-Laguerre in t = s - 1, 32 nodes: 1 + t_j, log(1 + t_j), log(lambda_j) - 1")
    parts.append(arr("lb_kq_hq32_s", [1 + a for a in t]))
    parts.append(arr("lb_kq_hq32_y", [mp.log(1 + a) for a in t]))
    parts.append(arr("lb_kq_hq32_c", [mp.log(a) - 1 for a in lam]))
    parts.append(arrq("lb_kq_hq32_y", [mp.log(1 + a) for a in t]))
    parts.append(arrq("lb_kq_hq32_c", [mp.log(a) - 1 for a in lam]))
    for N, s0 in ((10, 8), (20, 3), (8, 10)):
        t, lam = gauss_laguerre(N)
        tag = "hq%do%d" % (N, s0)
        parts.append("// one-slot rule: Gauss-Laguerre in t = s - %d, %d nodes: %d + t_j, log(%d + t_j), log(lambda_j) - %d"
                     % (s0, N, s0, s0, s0))
        parts.append(arr("lb_kq_%s_s" % tag, [s0 + a for a in t]))
        parts.append(arr("lb_kq_%s_y" % tag, [mp.log(s0 + a) for a in t]))
        parts.append(arr("lb_kq_%s_c" % tag, [mp.log(a) - s0 for a in lam]))
        parts.append(arrq("lb_kq_%s_y" % tag, [mp.log(s0 + a) for a in t]))
        parts.append(arrq("lb_kq_%s_c" % tag, [mp.log(a) - s0 for a in lam]))
    parts.append("// log 8, log 3 and log 10, the split points of the one-slot rules")
    for s0 in (8, 3, 10):
        parts.append("#define LB_KQ_LOG%d %r" % (s0, float(mp.log(s0))))
    for s0 in (8, 3, 10):
        parts.append("#define LB_KQ_LOG%d_Q53 %dll" % (s0, int(mp.nint(mp.log(s0) * mp.mpf(2) ** 53))))
    with open(out, "w") as f:
        f.write("\n".join(parts) + "\n")


if __name__ == "__main__":
    main()
