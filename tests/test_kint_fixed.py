"""The values' fixed-point K-integral sums (csrc/lb_kint.cuh), emulated on
the CPU with the host build of the integer-pipe helpers (csrc/lb_intmath.cuh)
and the Q53 rule tables (csrc/kquad_tables.h), against the oracle.

Per pair, as the kernel does it: v - 1/2 in Q58, gk = log beta (plus
(v + 1/2) log s0 for the one-slot rules) in Q53, each node's log term
L = C - S + (v - 1/2)(Y + log z) in Q53 with z = s + 2x, the shift m = max L,
the terms e^(L - m) in Q58 (Q56 for the rules with up to four nodes per lane)
summed as integers, and log K = prefactor + m + log(sum) (paper Sec. 3.2,
Eq. "log Kv integral" and Eq. "log sum trick").  The prefactor is taken in
40 digits here, so the test measures the integral's part: the rules'
truncation (at most 5e-17 for the one-slot rules, 2e-16 for the others,
test_kquad.py), the node positions s = s0 u^beta that the kernel forms in
double precision -- with beta rounded, beta (v + 1/2) = n holds only to
rounding, and the tables' u^(n-1) leaves a relative error of about
n (beta'/beta - 1) log u per node, up to 3.5e-16 of the scale at x near 1 --
and the fixed-point rounding; bound 4e-16 in the units of the error metric
for every rule (the end-to-end gate is 4e-15)."""
import os
import re

import numpy as np
import pytest

import oracle
from intmath_host import ix_exp, ix_exp_q58_fx, ix_fix, ix_log_q53, ix_mul_q58

mp = pytest.importorskip("mpmath")

TABLES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_2409_08729_gb300", "csrc",
                      "kquad_tables.h")


def _tables():
    txt = open(TABLES).read()
    t = {}
    for m in re.finditer(r"static __device__ const (double|long long) (\w+)\[(\d+)\] = \{([^}]*)\};", txt):
        vals = [v.strip() for v in m.group(4).replace("\n", " ").split(",") if v.strip()]
        if m.group(1) == "double":
            t[m.group(2)] = np.array([float(v) for v in vals])
        else:
            t[m.group(2)] = np.array([int(v[:-2]) for v in vals], dtype=np.int64)
    for m in re.finditer(r"#define (LB_KQ_\w+) (\S+)", txt):
        t[m.group(1)] = int(m.group(2)[:-2]) if m.group(2).endswith("ll") else float(m.group(2))
    return t


T = _tables()

# rule: (g nodes, h table, s0 of a one-slot rule or None); the s0 = 10 rule
# takes n = 6 (beta = 12/(2v+1)) and its own g constants
RULES = {
    "one, s0 = 8": (22, "hq10o8", 8),
    "one, s0 = 3": (12, "hq20o3", 3),
    "one, s0 = 10": (24, "hq8o10", 10),
    "g32+hl32": (32, "hl32", None),
    "g64+hl32": (64, "hl32", None),
    "g24+hl40": (24, "hl40", None),
    "g32+hq32": (32, "hq32", None),
}
CASES = {
    "one, s0 = 8": ([2.0, 2.37, 3.9, 5.5, 6.99], [1e-300, 1e-8, 0.0128, 0.3, 1.0, 4.7, 13.0, 25.0, 30.0]),
    "one, s0 = 3": ([7.0, 9.3, 12.71, 16.0], [1e-300, 1e-8, 0.0128, 0.3, 1.0, 4.7, 13.0, 25.0, 30.0]),
    "one, s0 = 10": ([0.9, 1.0, 1.3, 1.7, 1.999], [0.8, 1.0, 2.85, 4.7, 13.0, 18.5, 25.0, 30.0]),
    "g32+hl32": ([0.9, 1.0, 1.2], [0.25, 1.0, 7.3, 25.0, 30.0]),
    "g64+hl32": ([0.4, 0.55, 0.89], [1e-3, 0.01, 0.2]),
    "g24+hl40": ([1.21, 1.99, 3.3, 5.0], [1e-300, 1e-6, 0.04, 1.0, 9.0, 25.0]),
    "g32+hq32": ([5.01, 8.5, 16.0], [1e-300, 0.01, 1.0, 12.0, 25.0]),
}


def _fixed_terms(v, x, rule):
    """The rule's node log terms L (Q53), node arguments z = s + 2x, and the
    right shift of the Q58 terms (2 where a lane holds up to four terms)."""
    ng, htag, s0 = RULES[rule]
    vmq = int(ix_fix(np.array([v - 0.5]), 58)[0])
    beta = (12.0 if s0 == 10 else 16.0) / (2.0 * v + 1.0)
    gkq = int(ix_log_q53(np.array([beta]))[0])
    logu = T["lb_kq_g%d_logu" % ng]
    gc = T["lb_kq_g24n6_c_q"] if s0 == 10 else T["lb_kq_g%d_c_q" % ng]
    if s0 is not None:
        ls0q = T["LB_KQ_LOG%d_Q53" % s0]
        gkq += int(ix_mul_q58(np.array([vmq]), np.array([ls0q]))[0]) + ls0q
        s = ix_exp(beta * logu + T["LB_KQ_LOG%d" % s0])
    else:
        s = ix_exp(beta * logu)
    tx = 2.0 * x
    Lg = (gc + gkq - ix_fix(s, 53)
          + ix_mul_q58(np.full(ng, vmq, dtype=np.int64), ix_log_q53(tx + s)))
    hs = T["lb_kq_%s_s" % htag]
    Lh = T["lb_kq_%s_c_q" % htag] + ix_mul_q58(np.full(hs.size, vmq, dtype=np.int64),
                                               T["lb_kq_%s_y_q" % htag] + ix_log_q53(hs + tx))
    return np.concatenate([Lg, Lh]), np.concatenate([tx + s, hs + tx]), (0 if s0 is not None else 2)


def _fixed_log_integral(v, x, rule):
    """m + log(sum) of the rule in the kernel's fixed-point arithmetic, as
    an exact rational m plus a 40-digit log of the integer sum."""
    L, _, sh = _fixed_terms(v, x, rule)
    assert np.abs(L).max() < 2 ** 61                  # |L| < 2^8 in value: far inside Q53's range
    m = int(L.max())
    q = sum(int(t) >> sh for t in ix_exp_q58_fx(L - m))
    assert q < 2 ** 64
    return mp.mpf(m) / mp.mpf(2) ** 53 + mp.log(mp.mpf(q) / mp.mpf(2) ** (58 - sh))


@pytest.mark.parametrize("rule", list(RULES))
def test_fixed_point_sums_against_oracle(rule):
    vs, xs = CASES[rule]
    V, X = np.meshgrid(np.array(vs), np.array(xs), indexing="ij")
    V, X = V.ravel(), X.ravel()
    hi, lo = oracle.log_k(V, X, want_lo=True)
    c = oracle.error_scale("k", V, X)
    bound = 4e-16
    with mp.workdps(40):
        for v, x, h, l, cc in zip(V, X, hi, lo, c):
            vm, xm = mp.mpf(v), mp.mpf(x)
            pre = mp.log(mp.pi) / 2 - mp.loggamma(vm + mp.mpf(0.5)) - vm * mp.log(2 * xm) - xm
            err = float(abs(pre + _fixed_log_integral(v, x, rule) - (mp.mpf(h) + mp.mpf(l)))) / max(abs(h), cc)
            assert err < bound, (rule, v, x, err)


@pytest.mark.parametrize("rule", list(RULES))
def test_fixed_point_derivative_sums_against_oracle(rule):
    """The x-derivative from the same integer terms t_j: d/dx log K =
    -(v/x + 1) + (2v - 1) sum_j t_j / (s_j + 2x) / sum_j t_j (the weights in
    double precision, as the kernel forms them), against the oracle's Bessel
    ratio: below 4e-16 relative."""
    vs, xs = CASES[rule]
    V, X = np.meshgrid(np.array(vs), np.array(xs), indexing="ij")
    V, X = V.ravel(), X.ravel()
    ref = oracle.dlog_k_dx(V, X)
    for v, x, r in zip(V, X, ref):
        L, z, sh = _fixed_terms(v, x, rule)
        t = ix_exp_q58_fx(L - L.max()) >> np.uint64(sh)
        w1 = float(np.sum(t.astype(np.float64) / z))
        s0 = float(sum(int(u) for u in t))
        d = -(v / x + 1.0) + (2.0 * v - 1.0) * (w1 / s0)
        assert abs(d - r) <= 4e-16 * abs(r) + 1e-300, (rule, v, x, abs(d - r) / abs(r))


def test_fixed_point_shift_is_exact():
    """Any shift is exact in the log-sum-exp: moving every node's log term by
    the same Q53 amount moves m by exactly that amount and leaves the integer
    sum unchanged (the terms see only L - m)."""
    rng = np.random.default_rng(4)
    L = rng.integers(-(60 << 53), 60 << 53, 64, dtype=np.int64)
    for shift in (0, 1, -(7 << 50), (3 << 53) + 12345):
        Ls = L + shift
        q0 = ix_exp_q58_fx(L - L.max())
        q1 = ix_exp_q58_fx(Ls - Ls.max())
        assert np.array_equal(q0, q1)
