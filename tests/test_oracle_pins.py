"""Pins of the extended-precision oracle to facts outside itself (CPU only).

Each test checks the oracle against something it does not compute from:
arbitrary-precision library values (mpmath), closed forms, exact rational
brute force, the Wronskian and recurrence identities (which tie the
independent I and K evaluators together), asymptotic limits, and double-
precision library special cases (scipy).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50


def dd(hi, lo):
    return mp.mpf(hi) + mp.mpf(lo)


def test_constants():
    assert abs(dd(*oracle.dd_const(0)) - mp.log(2)) < mp.mpf(10) ** -32
    assert abs(dd(*oracle.dd_const(1)) - mp.pi) < mp.mpf(10) ** -32


@pytest.mark.parametrize("a", [-600.0, -80.5, -1.0, -1e-8, 0.0, 3e-9, 0.5, 1.0, 2.302585092994046, 37.25, 700.0])
def test_dd_exp(a):
    hi, lo = oracle.dd_exp(a, 0.0)
    ref = mp.exp(mp.mpf(a))
    assert abs(dd(hi, lo) / ref - 1) < mp.mpf(10) ** -29


@pytest.mark.parametrize("a", [1e-200, 1e-5, 0.3, 1.0 - 2 ** -40, 1.0, 1.0 + 2 ** -30, 2.0, 10.0, 1e5, 1e200])
def test_dd_log(a):
    hi, lo = oracle.dd_log(a, 0.0)
    ref = mp.log(mp.mpf(a))
    assert abs(dd(hi, lo) - ref) < mp.mpf(10) ** -30 * max(1, abs(ref))


@pytest.mark.parametrize("t", [1e-20, -3e-9, 2.5e-4, -9.9e-4, 0.5, 3.0])
def test_dd_log1p(t):
    hi, lo = oracle.dd_log1p(t, 0.0)
    ref = mp.log1p(mp.mpf(t))
    assert abs(dd(hi, lo) / ref - 1) < mp.mpf(10) ** -29


@pytest.mark.parametrize("n", [1, 2, 3, 7, 20, 39, 40, 41, 171, 1000, 100000])
def test_dd_lgamma_integers(n):
    """lgamma(n) = log((n-1)!) with the factorial formed exactly in integers."""
    hi, lo = oracle.dd_lgamma(float(n), 0.0)
    ref = mp.log(mp.mpf(math.factorial(n - 1))) if n < 3000 else mp.loggamma(n)
    assert abs(dd(hi, lo) - ref) < mp.mpf(10) ** -29 * max(1, abs(ref))


@pytest.mark.parametrize("n", [1, 2, 5, 19, 60])
def test_dd_lgamma_half_integers(n):
    """Gamma(n + 1/2) = (2n)! sqrt(pi) / (4^n n!)."""
    hi, lo = oracle.dd_lgamma(n + 0.5, 0.0)
    ref = mp.log(mp.mpf(math.factorial(2 * n)) * mp.sqrt(mp.pi) / (mp.mpf(4) ** n * math.factorial(n)))
    assert abs(dd(hi, lo) - ref) < mp.mpf(10) ** -29 * max(1, abs(ref))


def test_against_mpmath_random():
    """Random (v, x) over [1e-4, 300]^2 and integer orders: rounding-level agreement."""
    rng = np.random.default_rng(2024)
    n = 120
    v = np.exp(rng.uniform(np.log(1e-4), np.log(300), n))
    v[:15] = rng.integers(0, 6, 15)
    x = np.exp(rng.uniform(np.log(1e-4), np.log(300), n))
    li, lo_i = oracle.log_i(v, x, want_lo=True)
    lk, lo_k = oracle.log_k(v, x, want_lo=True)
    for j in range(n):
        # mpmath's K for large orders cancels internally (at 50 digits it returns a
        # negative K_208.56(138.45)); 150 working digits make it reliable here.
        with mp.workdps(150):
            ri = mp.log(mp.besseli(v[j], x[j]))
            rk = mp.log(mp.besselk(v[j], x[j]))
        assert abs(dd(li[j], lo_i[j]) - ri) <= mp.mpf(10) ** -26 * max(1, abs(ri)), (v[j], x[j])
        assert abs(dd(lk[j], lo_k[j]) - rk) <= mp.mpf(10) ** -26 * max(1, abs(rk)), (v[j], x[j])


@pytest.mark.parametrize("x", [1e-6, 0.01, 0.7, 2.0, 19.7, 100.0, 3000.0, 1e5])
def test_half_order_closed_forms(x):
    """I_{1/2}(x) = sqrt(2/(pi x)) sinh x; K_{1/2}(x) = sqrt(pi/(2x)) e^-x;
    K_{3/2}(x) = K_{1/2}(x) (1 + 1/x)."""
    X = mp.mpf(x)
    li = dd(*[a[0] for a in oracle.log_i([0.5], [x], want_lo=True)])
    lk = dd(*[a[0] for a in oracle.log_k([0.5], [x], want_lo=True)])
    lk3 = dd(*[a[0] for a in oracle.log_k([1.5], [x], want_lo=True)])
    ri = mp.log(mp.sqrt(2 / (mp.pi * X)) * mp.sinh(X))
    rk = mp.log(mp.sqrt(mp.pi / (2 * X))) - X
    assert abs(li - ri) < mp.mpf(10) ** -26 * max(1, abs(ri))
    assert abs(lk - rk) < mp.mpf(10) ** -26 * max(1, abs(rk))
    assert abs(lk3 - (rk + mp.log1p(1 / X))) < mp.mpf(10) ** -26 * max(1, abs(rk))


def _pairs(seed, n, vmax=1e4, xmin=1e-5, xmax=1e5):
    """Orders rounded to multiples of 2^-24 so that v +- 1 are exact doubles."""
    rng = np.random.default_rng(seed)
    v = np.exp(rng.uniform(np.log(1e-3), np.log(vmax), n))
    v = np.round(v * 2.0 ** 24) / 2.0 ** 24
    x = np.exp(rng.uniform(np.log(xmin), np.log(xmax), n))
    return v, x


def _dd_vals(fn, v, x):
    hi, lo = fn(v, x, want_lo=True)
    return [dd(a, b) for a, b in zip(hi, lo)]


def test_wronskian():
    """I_v K_{v+1} + I_{v+1} K_v = 1/x (DLMF 10.28.2): ties the series (I) and
    integral (K) evaluators, which share no code, to each other."""
    v, x = _pairs(7, 200)
    li0, li1 = _dd_vals(oracle.log_i, v, x), _dd_vals(oracle.log_i, v + 1, x)
    lk0, lk1 = _dd_vals(oracle.log_k, v, x), _dd_vals(oracle.log_k, v + 1, x)
    for j in range(v.size):
        a, b = li0[j] + lk1[j], li1[j] + lk0[j]
        m = max(a, b)
        lhs = m + mp.log(mp.exp(a - m) + mp.exp(b - m))
        rhs = -mp.log(mp.mpf(x[j]))
        assert abs(lhs - rhs) < mp.mpf(10) ** -24 * max(1, abs(a), abs(b)), (v[j], x[j])


def test_recurrences():
    """I_{v-1} = I_{v+1} + (2v/x) I_v and K_{v+1} = K_{v-1} + (2v/x) K_v (DLMF 10.29.1)."""
    v, x = _pairs(8, 150)
    v = v + 1.0
    lim, li0, lip = (_dd_vals(oracle.log_i, v + d, x) for d in (-1.0, 0.0, 1.0))
    lkm, lk0, lkp = (_dd_vals(oracle.log_k, v + d, x) for d in (-1.0, 0.0, 1.0))
    for j in range(v.size):
        c = mp.log(2 * mp.mpf(v[j]) / mp.mpf(x[j]))
        for lhs, t1, t2 in ((lim[j], lip[j], c + li0[j]), (lkp[j], lkm[j], c + lk0[j])):
            m = max(t1, t2)
            rhs = m + mp.log(mp.exp(t1 - m) + mp.exp(t2 - m))
            assert abs(lhs - rhs) < mp.mpf(10) ** -24 * max(1, abs(lhs)), (v[j], x[j])


@pytest.mark.parametrize("v", [0.0, 0.3, 1.0, 7.5, 120.0])
def test_small_argument_limits(v):
    """x -> 0: log I_v = v log(x/2) - lgamma(v+1) + x^2/(4(v+1)) + O(x^4);
    log K_v = lgamma(v) + v log(2/x) - log 2 + O(x^2) for v > 1, and
    log K_0 = log(-log(x/2) - gamma) + O(x^2 log x)."""
    x = 1e-9
    X = mp.mpf(x)
    li = mp.mpf(oracle.log_i([v], [x])[0])
    ref = v * mp.log(X / 2) - mp.loggamma(v + 1) + X ** 2 / (4 * (v + 1))
    assert abs(li - ref) <= 1e-16 * max(1, abs(ref))
    lk = mp.mpf(oracle.log_k([v], [x])[0])
    if v > 1:
        refk = mp.loggamma(v) + v * mp.log(2 / X) - mp.log(2)
        assert abs(lk - refk) <= 1e-14 * max(1, abs(refk))
    elif v == 0:
        refk = mp.log(-mp.log(X / 2) - mp.euler)
        assert abs(lk - refk) <= 1e-14


@pytest.mark.parametrize("v", [0.0, 0.5, 2.0, 10.0])
def test_large_argument_limit(v):
    """x -> inf: log I_v(x) = x - log(2 pi x)/2 - (4v^2 - 1)/(8x) + O(x^-2),
    log K_v(x) = log(pi/(2x))/2 - x + (4v^2 - 1)/(8x) + O(x^-2)."""
    x = 1e7
    X = mp.mpf(x)
    mu = 4 * mp.mpf(v) ** 2
    li = mp.mpf(oracle.log_i([v], [x])[0])
    lk = mp.mpf(oracle.log_k([v], [x])[0])
    ri = X - mp.log(2 * mp.pi * X) / 2 - (mu - 1) / (8 * X)
    rk = mp.log(mp.pi / (2 * X)) / 2 - X + (mu - 1) / (8 * X)
    bound = (abs(mu - 1) * abs(mu - 9) + 1) / (64 * X ** 2) + 1e-16 * X
    assert abs(li - ri) <= bound
    assert abs(lk - rk) <= bound


@pytest.mark.parametrize("n", [0, 1, 2, 5])
@pytest.mark.parametrize("x", [Fraction(1, 3), Fraction(1, 2), Fraction(2), Fraction(7, 2)])
def test_brute_force_exact_series(n, x):
    """Integer order, rational argument: I_n(x) = sum (x/2)^(2k+n) / (k! (k+n)!)
    summed exactly in rationals until the terms fall below 1e-45."""
    x = Fraction(float(x))          # the double the oracle receives, exactly
    s = Fraction(0)
    k = 0
    while True:
        term = (x / 2) ** (2 * k + n) / (math.factorial(k) * math.factorial(k + n))
        s += term
        if term < Fraction(1, 10 ** 45) * s:
            break
        k += 1
    ref = mp.log(mp.mpf(s.numerator) / s.denominator)
    hi, lo = oracle.log_i([float(n)], [float(x)], want_lo=True)
    assert abs(dd(hi[0], lo[0]) - ref) < mp.mpf(10) ** -28 * max(1, abs(ref))


def test_scipy_integer_orders():
    """Orders 0 and 1 against scipy's exponentially scaled i0e, i1e, k0e, k1e."""
    special = pytest.importorskip("scipy.special")
    x = np.exp(np.linspace(np.log(1e-3), np.log(700.0), 400))
    for v, fi, fk in ((0.0, special.i0e, special.k0e), (1.0, special.i1e, special.k1e)):
        ri = np.log(fi(x)) + x
        rk = np.log(fk(x)) - x
        oi = oracle.log_i(np.full_like(x, v), x)
        ok = oracle.log_k(np.full_like(x, v), x)
        assert np.max(np.abs(oi - ri) / np.maximum(1, np.abs(ri))) < 2e-15
        assert np.max(np.abs(ok - rk) / np.maximum(1, np.abs(rk))) < 2e-15


def test_derivatives_against_mpmath():
    rng = np.random.default_rng(9)
    v = np.exp(rng.uniform(np.log(1e-3), np.log(200), 40))
    x = np.exp(rng.uniform(np.log(1e-3), np.log(300), 40))
    di = oracle.dlog_i_dx(v, x)
    dk = oracle.dlog_k_dx(v, x)
    for j in range(v.size):
        with mp.workdps(150):
            ri = mp.besseli(v[j], x[j], derivative=1) / mp.besseli(v[j], x[j])
            rk = mp.diff(lambda t: mp.log(mp.besselk(v[j], t)), x[j])
        assert abs(di[j] - ri) <= 4e-16 * abs(ri), (v[j], x[j])
        assert abs(dk[j] - rk) <= 4e-16 * abs(rk), (v[j], x[j])


def test_order_derivative_central_difference():
    v = np.array([0.5, 3.0, 40.0])
    x = np.array([2.0, 10.0, 30.0])
    dv = oracle.dlog_i_dv(v, x)
    for j in range(v.size):
        ref = mp.diff(lambda t: mp.log(mp.besseli(t, x[j])), v[j])
        assert abs(dv[j] - ref) <= 1e-8 * abs(ref)


def test_vmf_log_normaliser():
    d = np.array([3.0, 2048.0, 8192.0, 32768.0])
    kappa = np.array([2.5, 300.0, 1600.0, 6700.0])
    got = oracle.vmf_log_c(d, kappa)
    for j in range(d.size):
        nu = mp.mpf(d[j]) / 2 - 1
        ref = nu * mp.log(kappa[j]) - mp.mpf(d[j]) / 2 * mp.log(2 * mp.pi) - mp.log(mp.besseli(nu, kappa[j]))
        assert abs(got[j] - ref) <= 1e-15 * max(1, abs(ref))
    # d = 3: C_3(k) = k / (4 pi sinh k) in closed form
    assert abs(got[0] - (math.log(2.5) - math.log(4 * math.pi * math.sinh(2.5)))) < 1e-14


def test_domain_edges():
    inf, nan = np.inf, np.nan
    v = np.array([0.0, 2.0, -1.0, 1.0, 1.0, inf, nan, inf])
    x = np.array([0.0, 0.0, 1.0, -1.0, inf, 1.0, 1.0, inf])
    li = oracle.log_i(v, x)
    assert li[0] == 0.0 and li[1] == -inf and np.isnan(li[2]) and np.isnan(li[3])
    assert li[4] == inf and li[5] == -inf and np.isnan(li[6]) and np.isnan(li[7])
    lk = oracle.log_k(v, x)
    assert lk[0] == inf and lk[1] == inf and np.isfinite(lk[2]) and np.isnan(lk[3])
    assert lk[4] == -inf and lk[5] == inf and np.isnan(lk[6]) and np.isnan(lk[7])
    # K is even in v
    assert oracle.log_k([-2.5], [3.0])[0] == oracle.log_k([2.5], [3.0])[0]


def test_error_metric():
    got = np.array([1.0, 2.0, np.inf, np.nan, 5.0])
    ref = np.array([1.0 + 1e-15, 2.0, np.inf, np.nan, np.nan])
    e = oracle.rel_err(got, ref, np.ones(5))
    assert e[0] == pytest.approx(1e-15, rel=1e-3) and e[1] == 0 and e[2] == 0 and e[3] == 0
    assert e[4] == np.inf


@pytest.mark.parametrize("v", [0.0, 0.3, 2.5, 1e5])
@pytest.mark.parametrize("x", [1e-300, 1e-200, 1e-6])
def test_extreme_small_arguments(v, x):
    """K at arguments where x cosh t overflows inside the integration range
    (the integrand is 0 there), and I at tiny x; mpmath at 60 digits."""
    with mp.workdps(60):
        rk = mp.log(mp.besselk(v, mp.mpf(x)))
        ri = mp.log(mp.besseli(v, mp.mpf(x)))
    lk = oracle.log_k([v], [x])[0]
    li = oracle.log_i([v], [x])[0]
    assert abs(lk - rk) <= 2e-16 * max(1, abs(rk))
    assert abs(li - ri) <= 2e-16 * max(1, abs(ri))
