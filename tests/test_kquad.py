"""The Gauss rules of the K integral (kquad_tables.h), checked on the CPU.

Each rule is summed the way lb_kint.cuh sums it, in 30-digit arithmetic from
the double-precision table entries, and log K built from the prefactor of
Rothwell's representation (paper Sec. 3.2):

  log K_v(x) = log(pi)/2 - lgamma(v + 1/2) - v log(2x) - x + log int_0^inf F(s) ds,
  F(s) = e^{-s} (s (s + 2x))^(v-1/2),

against the oracle (double-double).  The error, in the units of the error
metric (|err| / max(|log K|, c), c = max(1, |x d/dx log K|, |v d/dv log K|)),
is the rule's truncation error plus the rounding of its table entries: what
the kernel would reach in exact arithmetic.  Bounds are 2e-16, a fifth of
the measured FP64 end-to-end maxima (rounding dominates), and 5e-17 for the
one-slot rules, whose error map was drawn at 1.5e-17.
"""
import os
import re

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = os.path.join(HERE, "..", "paper_2409_08729_gb300", "csrc", "kquad_tables.h")


def _tables():
    txt = open(TABLES).read()
    out = {}
    for m in re.finditer(r"static __device__ const double (\w+)\[(\d+)\] = \{([^}]*)\};", txt):
        vals = [float(t) for t in m.group(3).replace("\n", " ").split(",") if t.strip()]
        assert len(vals) == int(m.group(2)), m.group(1)
        out[m.group(1)] = vals
    for m in re.finditer(r"static __device__ const long long (\w+)\[(\d+)\] = \{([^}]*)\};", txt):
        vals = [int(t.strip()[:-2]) for t in m.group(3).replace("\n", " ").split(",") if t.strip()]
        assert len(vals) == int(m.group(2)), m.group(1)
        out[m.group(1)] = vals
    for m in re.finditer(r"#define (LB_KQ_\w+) (\S+)", txt):
        out[m.group(1)] = int(m.group(2)[:-2]) if m.group(2).endswith("ll") else float(m.group(2))
    return out


T = _tables()


def _tab(name, q):
    """A table of log terms: the double entries, or (q) the Q53 ones that
    the values' fixed-point node sums use, as exact rationals."""
    if q:
        return [mp.mpf(t) / mp.mpf(2) ** 53 for t in T[name + "_q"]]
    return T[name]


def _g_fixed(v, x, N, q=False):
    """beta sum_j e^{c_j + (v-1/2) log(2x + u_j^beta) - u_j^beta} (s = u^beta on [0, 1])."""
    beta = mp.mpf(16) / (2 * v + 1)
    tot = mp.mpf(0)
    for lu, c in zip(T["lb_kq_g%d_logu" % N], _tab("lb_kq_g%d_c" % N, q)):
        ub = mp.exp(beta * lu)
        tot += mp.exp(c + (v - mp.mpf(0.5)) * mp.log(2 * x + ub) - ub)
    return beta * tot


def _h(v, x, tag, q=False):
    """sum_j e^{c_j + (v-1/2)(y_j + log(s_j + 2x))} for the h table `tag`."""
    tot = mp.mpf(0)
    for s, y, c in zip(T["lb_kq_%s_s" % tag], _tab("lb_kq_%s_y" % tag, q), _tab("lb_kq_%s_c" % tag, q)):
        tot += mp.exp(c + (v - mp.mpf(0.5)) * (y + mp.log(s + 2 * x)))
    return tot


def _g_one(v, x, N, ls0, q=False, n=8):
    """The [0, s0] part of a one-slot rule: s_j = e^{beta log u_j + log s0},
    beta = 2n/(2v+1) (n = 8, or 6 for the rule with s0 = 10)."""
    beta = mp.mpf(2 * n) / (2 * v + 1)
    ctab = "lb_kq_g%d_c" % N if n == 8 else "lb_kq_g%dn%d_c" % (N, n)
    tot = mp.mpf(0)
    for lu, c in zip(T["lb_kq_g%d_logu" % N], _tab(ctab, q)):
        s = mp.exp(beta * lu + ls0)
        tot += mp.exp(c + (v + mp.mpf(0.5)) * ls0 + (v - mp.mpf(0.5)) * mp.log(2 * x + s) - s)
    return beta * tot


def _ls0(name, q):
    return mp.mpf(T[name + "_Q53"]) / mp.mpf(2) ** 53 if q else mp.mpf(T[name])


RULES = {
    # name: (sum of the rule, the orders and arguments it serves)
    "g32+hl32": (lambda v, x, q: _g_fixed(v, x, 32, q) + _h(v, x, "hl32", q), [0.9, 0.97, 1.0, 1.2],
                 [0.25, 1.0, 7.3, 25.0, 30.0]),
    "g64+hl32": (lambda v, x, q: _g_fixed(v, x, 64, q) + _h(v, x, "hl32", q), [0.4, 0.55, 0.89], [1e-3, 0.01, 0.2]),
    "g24+hl40": (lambda v, x, q: _g_fixed(v, x, 24, q) + _h(v, x, "hl40", q), [1.21, 1.5, 1.99, 3.3, 5.0],
                 [1e-300, 1e-6, 0.04, 1.0, 9.0, 25.0]),
    "g32+hq32": (lambda v, x, q: _g_fixed(v, x, 32, q) + _h(v, x, "hq32", q), [5.01, 8.5, 16.0],
                 [1e-300, 0.01, 1.0, 12.0, 25.0]),
    "one, s0 = 8": (lambda v, x, q: _g_one(v, x, 22, _ls0("LB_KQ_LOG8", q), q) + _h(v, x, "hq10o8", q),
                    [2.0, 2.37, 3.9, 5.5, 6.99], [1e-300, 1e-8, 0.0128, 0.3, 1.0, 4.7, 13.0, 25.0, 30.0]),
    "one, s0 = 3": (lambda v, x, q: _g_one(v, x, 12, _ls0("LB_KQ_LOG3", q), q) + _h(v, x, "hq20o3", q),
                    [7.0, 7.9, 9.3, 12.71, 16.0, 16.5], [1e-300, 1e-8, 0.0128, 0.3, 1.0, 4.7, 13.0, 25.0, 30.0]),
    "one, s0 = 10": (lambda v, x, q: _g_one(v, x, 24, _ls0("LB_KQ_LOG10", q), q, n=6) + _h(v, x, "hq8o10", q),
                     [0.9, 0.95, 1.0, 1.3, 1.5, 1.8, 1.999], [0.8, 1.0, 1.6, 2.85, 4.7, 9.0, 13.0, 18.5, 25.0, 30.0]),
}


@pytest.mark.parametrize("q", [False, True], ids=["double tables", "Q53 tables"])
@pytest.mark.parametrize("name", list(RULES))
def test_rule_error_map(name, q):
    fn0, vs, xs = RULES[name]
    fn = lambda v, x: fn0(v, x, q)
    V, X = np.meshgrid(np.array(vs), np.array(xs), indexing="ij")
    V, X = V.ravel(), X.ravel()
    hi, lo = oracle.log_k(V, X, want_lo=True)
    c = oracle.error_scale("k", V, X)
    worst = 0.0
    with mp.workdps(30):
        for v, x, h, l, cc in zip(V, X, hi, lo, c):
            vm, xm = mp.mpf(v), mp.mpf(x)
            lk = (mp.log(mp.pi) / 2 - mp.loggamma(vm + mp.mpf(0.5)) - vm * mp.log(2 * xm) - xm
                  + mp.log(fn(vm, xm)))
            err = float(abs(lk - (mp.mpf(h) + mp.mpf(l)))) / max(abs(h), cc)
            worst = max(worst, err)
            # the s0 = 10 rule (v < 2, x <= 30) always runs from the Q53 tables
            # (the double ones serve only pairs past v = 16.5 or x = 32)
            bound = 5e-17 if name.startswith("one") and (q or name != "one, s0 = 10") else 2e-16
            assert err < bound, (name, v, x, err)
    assert worst > 0.0


def test_q53_tables():
    """Every Q53 table (the log terms of the values' fixed-point node sums)
    and the Q53 split-point logarithms hold the same 40-digit values as their
    double twins: within half a unit of 2^-53 plus half an ulp of the double."""
    names = [k[:-2] for k in T if k.endswith("_q")]
    assert len(names) == 20
    with mp.workdps(40):
        for n in names:
            for d, qv in zip(T[n], T[n + "_q"]):
                err = abs(mp.mpf(qv) / mp.mpf(2) ** 53 - mp.mpf(d))
                assert err <= mp.mpf(2) ** -54 + mp.mpf(np.spacing(abs(d))) / 2, n
        for n in ("LB_KQ_LOG8", "LB_KQ_LOG3", "LB_KQ_LOG10"):
            err = abs(mp.mpf(T[n + "_Q53"]) / mp.mpf(2) ** 53 - mp.mpf(T[n]))
            assert err <= mp.mpf(2) ** -54 + mp.mpf(np.spacing(T[n])) / 2, n


def test_one_slot_tables():
    """The one-slot rules' tables: node counts and the split points."""
    assert len(T["lb_kq_g22_logu"]) == 22 and len(T["lb_kq_hq10o8_s"]) == 10
    assert len(T["lb_kq_g12_logu"]) == 12 and len(T["lb_kq_hq20o3_s"]) == 20
    assert T["LB_KQ_LOG8"] == float(mp.log(8)) and T["LB_KQ_LOG3"] == float(mp.log(3))
    # the Laguerre nodes start past the split point; weights sum to e^{-s0}
    for tag, s0 in (("hq10o8", 8), ("hq20o3", 3)):
        assert min(T["lb_kq_%s_s" % tag]) > s0
        w = sum(mp.exp(c) for c in T["lb_kq_%s_c" % tag])
        assert abs(w / mp.exp(-s0) - 1) < 1e-15


def _g_fixed_dx(v, x, N):
    """The g part of a fixed rule and of its x-derivative's weighted sum:
    (beta sum_j F_j, beta sum_j F_j / (s_j + 2x))."""
    beta = mp.mpf(16) / (2 * v + 1)
    s0 = s1 = mp.mpf(0)
    for lu, c in zip(T["lb_kq_g%d_logu" % N], T["lb_kq_g%d_c" % N]):
        ub = mp.exp(beta * lu)
        t = mp.exp(c + (v - mp.mpf(0.5)) * mp.log(2 * x + ub) - ub)
        s0 += t
        s1 += t / (ub + 2 * x)
    return beta * s0, beta * s1


def _h_dx(v, x, tag):
    s0 = s1 = mp.mpf(0)
    for s, y, c in zip(T["lb_kq_%s_s" % tag], T["lb_kq_%s_y" % tag], T["lb_kq_%s_c" % tag]):
        t = mp.exp(c + (v - mp.mpf(0.5)) * (y + mp.log(s + 2 * x)))
        s0 += t
        s1 += t / (s + 2 * x)
    return s0, s1


# The x-derivative's fixed and packed rules (the one-slot rules: below):
# d/dx log K = -(v/x + 1) + (2v - 1) <1/(s + 2x)>, the mean weighted by
# F over the nodes (dF/dx = F (2v - 1)/(s + 2x)), with the orders and
# arguments each rule serves, including the small orders at 0.25 <= x < 0.6
# that take 64 g nodes for the derivative.
DX_RULES = {
    "g32+hl32": ((32, "hl32"), [0.0, 0.05, 0.1, 0.5, 0.9, 1.0, 1.2], [0.6, 1.0, 3.0, 7.3, 25.0, 30.0]),
    "g32+hl32 (v >= 0.1)": ((32, "hl32"), [0.1, 0.3, 0.5, 0.8, 0.89], [0.25, 0.3, 0.45]),
    "g64+hl32": ((64, "hl32"), [0.0, 1e-3, 0.05, 0.099], [5e-3, 0.01, 0.1, 0.25, 0.3, 0.45, 0.59]),
    "g64+hl32 (x < 0.25)": ((64, "hl32"), [0.4, 0.55, 0.89], [1e-3, 0.01, 0.05, 0.2]),
    "g24+hl40": ((24, "hl40"), [1.21, 1.5, 2.5, 3.3, 5.0], [1e-300, 1e-6, 0.04, 1.0, 9.0, 25.0]),
    "g32+hq32": ((32, "hq32"), [5.01, 8.5, 12.0, 16.0], [1e-300, 1e-8, 0.01, 1.0, 12.0, 25.0]),
}


@pytest.mark.parametrize("name", list(DX_RULES))
def test_derivative_rule_error_map(name):
    """Each derivative rule, summed from its double table entries in 30-digit
    arithmetic, against the oracle's d/dx log K (the Bessel ratio of DLMF
    10.29.2): relative error below 2e-16 (worst measured: 1.2e-16)."""
    (N, tag), vs, xs = DX_RULES[name]
    V, X = np.meshgrid(np.array(vs), np.array(xs), indexing="ij")
    V, X = V.ravel(), X.ravel()
    ref = oracle.dlog_k_dx(V, X)
    with mp.workdps(30):
        for v, x, r in zip(V, X, ref):
            vm, xm = mp.mpf(v), mp.mpf(x)
            a0, a1 = _g_fixed_dx(vm, xm, N)
            b0, b1 = _h_dx(vm, xm, tag)
            d = -(vm / xm + 1) + (2 * vm - 1) * (a1 + b1) / (a0 + b0)
            err = float(abs(d - mp.mpf(r)) / abs(mp.mpf(r)))
            assert err < 2e-16, (name, v, x, err)


def _one_dx(v, x, N, htag, ls0, n=8):
    """A one-slot rule and its x-derivative's weighted sum (s = s0 u^beta on [0, s0])."""
    beta = mp.mpf(2 * n) / (2 * v + 1)
    a0 = a1 = mp.mpf(0)
    for lu, c in zip(T["lb_kq_g%d_logu" % N], T["lb_kq_g%d_c" % N if n == 8 else "lb_kq_g%dn%d_c" % (N, n)]):
        s = mp.exp(beta * lu + ls0)
        t = mp.exp(c + (v + mp.mpf(0.5)) * ls0 + (v - mp.mpf(0.5)) * mp.log(2 * x + s) - s)
        a0 += beta * t
        a1 += beta * t / (s + 2 * x)
    b0, b1 = _h_dx(v, x, htag)
    return a0 + b0, a1 + b1


@pytest.mark.parametrize("rule", ["s0 = 8", "s0 = 3", "s0 = 10"])
def test_derivative_one_slot_rules(rule):
    """The one-slot rules serve the x-derivative too (2 <= v <= 16.5): their
    weighted mean of 1/(s + 2x), summed from the double tables in 30 digits,
    against the oracle's d/dx log K, below 2e-16 relative (the map over
    x in [1e-300, 30] measured at most 1.1e-16, the reference's own
    rounding)."""
    n = 8
    xs = [1e-300, 1e-8, 1e-3, 0.0128, 0.3, 1.0, 4.7, 13.0, 25.0, 30.0]
    if rule == "s0 = 8":
        N, tag, ls0, vs = 22, "hq10o8", mp.mpf(T["LB_KQ_LOG8"]), [2.0, 2.2, 3.9, 5.5, 6.99]
    elif rule == "s0 = 3":
        N, tag, ls0, vs = 12, "hq20o3", mp.mpf(T["LB_KQ_LOG3"]), [7.0, 9.3, 12.71, 16.0, 16.5]
    else:                                          # 0.9 <= v < 2, x >= 0.8
        N, tag, ls0, vs, n = 24, "hq8o10", mp.mpf(T["LB_KQ_LOG10"]), [0.9, 1.0, 1.3, 1.7, 1.999], 6
        xs = [0.8, 1.0, 1.6, 4.7, 9.0, 18.5, 25.0, 30.0]
    V, X = np.meshgrid(np.array(vs), np.array(xs), indexing="ij")
    V, X = V.ravel(), X.ravel()
    ref = oracle.dlog_k_dx(V, X)
    with mp.workdps(30):
        for v, x, r in zip(V, X, ref):
            vm, xm = mp.mpf(v), mp.mpf(x)
            a0, a1 = _one_dx(vm, xm, N, tag, ls0, n)
            d = -(vm / xm + 1) + (2 * vm - 1) * a1 / a0
            err = float(abs(d - mp.mpf(r)) / abs(mp.mpf(r)))
            assert err < 2e-16, (rule, v, x, err)


def test_derivative_needs_64_nodes_below_x_0_6():
    """The reason for the derivative's boundary: at v = 0, x = 0.25 the 32-node
    g rule leaves ~7e-15 in d/dx log K, the 64-node rule < 1e-16."""
    v, x = 0.0, 0.25
    ref = oracle.dlog_k_dx(np.array([v]), np.array([x]))[0]
    with mp.workdps(30):
        vm, xm = mp.mpf(v), mp.mpf(x)
        errs = []
        for N in (32, 64):
            a0, a1 = _g_fixed_dx(vm, xm, N)
            b0, b1 = _h_dx(vm, xm, "hl32")
            d = -(vm / xm + 1) + (2 * vm - 1) * (a1 + b1) / (a0 + b0)
            errs.append(float(abs(d - mp.mpf(ref)) / abs(mp.mpf(ref))))
    assert errs[0] > 1e-15 and errs[1] < 1e-16


def _split_dx_above_1e3(v, x):
    """The split g rule for 1e-3 <= x < 5e-3 (y1 = log(128 x) > -4, so of its
    log-s panels only [y1, 0] is non-empty): 64 nodes on [0, s1], s = s1 u^beta,
    16 Gauss-Legendre nodes in y = log s on [y1, 0], the 32 h nodes; the
    derivative's weighted sums as in _g_fixed_dx."""
    beta = mp.mpf(16) / (2 * v + 1)
    s1 = 128 * x
    y1 = mp.log(s1)
    s0 = s1w = mp.mpf(0)
    for lu, c in zip(T["lb_kq_g64_logu"], T["lb_kq_g64_c"]):
        r = mp.exp(beta * lu)
        s = s1 * r
        t = beta * mp.exp(2 * v * y1 + c + (v - mp.mpf(0.5)) * mp.log(r + mp.mpf(1) / 64) - s)
        s0 += t
        s1w += t / (s + 2 * x)
    for tt, lw in zip(T["lb_kq_gl16_t"], T["lb_kq_gl16_logw"]):
        y = y1 * (1 - tt)
        s = mp.exp(y)
        t = mp.exp(lw + mp.log(-y1) + (v + mp.mpf(0.5)) * y + (v - mp.mpf(0.5)) * mp.log(s + 2 * x) - s)
        s0 += t
        s1w += t / (s + 2 * x)
    h0, h1 = _h_dx(v, x, "hl32")
    return -(v / x + 1) + (2 * v - 1) * (s1w + h1) / (s0 + h0)


def test_derivative_split_rule_up_to_5e_3():
    """For v < 0.1 the derivative takes the split rule up to x = 5e-3, where
    the 64-node rule leaves 8e-15 (v = 0, x = 1e-3): the split rule's error
    there is below 2e-16."""
    with mp.workdps(30):
        for v in (0.0, 1e-4, 0.01, 0.05, 0.099):
            for x in (1e-3, 1.5e-3, 2e-3, 3e-3, 4.9e-3):
                ref = oracle.dlog_k_dx(np.array([v]), np.array([x]))[0]
                d = _split_dx_above_1e3(mp.mpf(v), mp.mpf(x))
                err = float(abs(d - mp.mpf(ref)) / abs(mp.mpf(ref)))
                assert err < 2e-16, (v, x, err)
        a0, a1 = _g_fixed_dx(mp.mpf(0), mp.mpf(1e-3), 64)
        b0, b1 = _h_dx(mp.mpf(0), mp.mpf(1e-3), "hl32")
        d64 = -(mp.mpf(1e-3) ** -1 * 0 + 1) - (a1 + b1) / (a0 + b0)
        ref = oracle.dlog_k_dx(np.array([0.0]), np.array([1e-3]))[0]
        assert float(abs(d64 - mp.mpf(ref)) / abs(mp.mpf(ref))) > 1e-15
