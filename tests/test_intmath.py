"""Integer-pipe exp and log (csrc/lb_intmath.cuh), host build, against the
oracle's double-double exp and log: within 0.51 ulp of the exact value."""
import numpy as np
import pytest

import oracle
from fractions import Fraction

from intmath_host import ix_exp, ix_exp_q58, ix_exp_q58_fx, ix_fix, ix_log, ix_log_q53, ix_mul_q58, ix_rcp, ix_rsqrt


def _ref(fn, a):
    out = np.empty((a.size, 2))
    for i, v in enumerate(a):
        out[i] = fn(float(v))
    return out


def _ulp_err(got, ref):
    return np.abs((got - ref[:, 0]) - ref[:, 1]) / np.spacing(np.abs(ref[:, 0]))


def test_exp_accuracy():
    rng = np.random.default_rng(11)
    y = np.concatenate([rng.uniform(-708, 708, 20000), rng.uniform(-1, 1, 5000), rng.uniform(-1e-3, 1e-3, 2000),
                        np.exp(rng.uniform(-40, 3, 3000)) * rng.choice([-1.0, 1.0], 3000),
                        np.log(2.0) / 512 * (np.arange(-600, 600) + 0.5),        # reduction boundaries
                        [0.5, -0.5, np.log(2.0), -np.log(2.0), 700.0, -700.0, 708.0, -708.0]])
    e = _ulp_err(ix_exp(y), _ref(oracle.dd_exp, y))
    assert e.max() < 0.51, (e.max(), y[e.argmax()])


def test_exp_special():
    got = ix_exp(np.array([0.0, -0.0, 1e-300, -1e-300, 2.0 ** -70, -708.5, -745.0, -1e300, 708.5]))
    assert list(got[:5]) == [1.0] * 5
    assert list(got[5:8]) == [0.0] * 3
    assert got[8] == np.inf


def test_log_accuracy():
    rng = np.random.default_rng(12)
    z = np.concatenate([np.exp(rng.uniform(-708, 709, 20000)), rng.uniform(0.5, 2.0, 5000),
                        1.0 + rng.uniform(-1e-3, 1e-3, 2000), 1.0 + rng.uniform(-1e-9, 1e-9, 1000),
                        1.0 + np.arange(1, 200) * 2.0 ** -52, 1.0 - np.arange(1, 200) * 2.0 ** -53,
                        1.0 + np.arange(512) / 512.0, 2.0 ** np.arange(-1022, 1024, 37),
                        [2.0 ** -1022, 1.7976931348623157e308, 3.0, 10.0, np.e]])
    ref = _ref(oracle.dd_log, z)
    e = _ulp_err(ix_log(z), ref)
    assert e.max() < 0.51, (e.max(), z[e.argmax()])


def test_results_next_to_powers_of_two():
    """Results just below and above a power of two (the rounding carry of the
    53-bit significand into the exponent)."""
    k = np.arange(-12, 10)
    nudge = np.array([-3, -2, -1, 0, 1, 2, 3])
    z = np.exp(2.0 ** k)[:, None] * (1.0 + nudge[None, :] * 2.0 ** -52)
    z = np.concatenate([z.ravel(), [np.nextafter(np.e, 0), np.nextafter(np.e, 4)]])
    e = _ulp_err(ix_log(z), _ref(oracle.dd_log, z))
    assert e.max() < 0.51, (e.max(), z[e.argmax()])
    y = (np.arange(-1000, 1000) * np.log(2.0))[:, None] * (1.0 + nudge[None, :] * 2.0 ** -52)
    y = y.ravel()
    y = y[np.abs(y) <= 708]
    e = _ulp_err(ix_exp(y), _ref(oracle.dd_exp, y))
    assert e.max() < 0.51, (e.max(), y[e.argmax()])


def test_log_special():
    got = ix_log(np.array([1.0, 2.0, 0.5, 0.0, -1.0, np.inf, 5e-324]))
    assert got[0] == 0.0
    assert got[1] == np.log(2.0) and got[2] == -np.log(2.0)
    assert got[3] == -np.inf and np.isnan(got[4]) and got[5] == np.inf
    assert got[6] == np.log(5e-324)          # subnormal: the libm log


@pytest.mark.parametrize("seed", [0, 1])
def test_exp_log_roundtrip(seed):
    """log(exp(y)) returns y to within the rounding of exp (|y| <= 700)."""
    rng = np.random.default_rng(seed)
    y = rng.uniform(-700, 700, 20000)
    back = ix_log(ix_exp(y))
    assert np.max(np.abs(back - y) / np.maximum(np.abs(y), 1.0)) < 4e-16


def test_exp_q58():
    """e^y in Q58 fixed point: within 0.6 units of 2^-58 of the exact value
    (double-double reference, summed exactly as fractions), y in [-45, ln 2)."""
    rng = np.random.default_rng(13)
    y = np.concatenate([rng.uniform(-45, 0.69, 3000), rng.uniform(-1, 0.01, 2000), -np.exp(rng.uniform(-70, 3, 1000)),
                        np.log(2.0) / 512 * (np.arange(-600, 200) + 0.5), -np.arange(36, 46, 0.25),
                        [0.0, -0.0, 2.0 ** -70, -2.0 ** -70, 0.5, -42.0, np.nextafter(-42.0, 0)]])
    got = ix_exp_q58(y)
    scale = Fraction(2) ** 58
    for yi, g in zip(y, got):
        hi, lo = oracle.dd_exp(float(yi))
        exact = (Fraction(hi) + Fraction(lo)) * scale
        assert abs(Fraction(int(g)) - exact) <= Fraction(6, 10), (yi, int(g), float(exact))
    assert int(got[-7]) == 2 ** 58 and int(got[-6]) == 2 ** 58


def test_exp_q58_sums():
    """32 terms e^(L - max L) summed in Q58 (as the K-integral warp sums do)
    match the double-double sum to 32 x 0.6 units of 2^-58."""
    rng = np.random.default_rng(14)
    for _ in range(50):
        L = rng.normal(0, 8, 32)
        y = L - L.max()
        got = sum(int(t) for t in ix_exp_q58(y))
        assert got < 2 ** 64
        exact = sum((Fraction(h) + Fraction(l)) for h, l in (oracle.dd_exp(float(v)) for v in y)) * Fraction(2) ** 58
        assert abs(got - exact) <= 32 * Fraction(6, 10)


def _ulp_err_exact(got, exact):
    """|got - exact| in ulps of exact (exact a Fraction)."""
    e = abs(Fraction(got) - exact)
    return float(e / Fraction(np.spacing(float(exact))))


def _args(seed):
    rng = np.random.default_rng(seed)
    z = np.concatenate([np.exp(rng.uniform(-700, 700, 4000)), rng.uniform(1.0, 2.0, 3000),
                        1.0 + np.arange(512) / 512.0, 1.0 + (np.arange(512) + 1) / 512.0 - 2.0 ** -52,
                        1.0 + np.arange(1, 100) * 2.0 ** -52, 2.0 - np.arange(1, 100) * 2.0 ** -52,
                        2.0 ** np.arange(-1022, 1022, 11), 3.0 * 2.0 ** np.arange(-1000, 1000, 13),
                        [2.0 ** -1022, np.nextafter(2.0 ** 1022, 0), 3.0, 10.0, 0.1, 1e300]])
    return z


def test_rcp_accuracy():
    """Integer-pipe 1/z within 0.51 ulp of the exact rational."""
    z = _args(15)
    got = ix_rcp(z)
    worst = max(_ulp_err_exact(g, 1 / Fraction(float(v))) for g, v in zip(got, z))
    assert worst < 0.51, worst


def test_rsqrt_accuracy():
    """Integer-pipe 1/sqrt(z) within 0.52 ulp (50-digit reference)."""
    mp = pytest.importorskip("mpmath")
    z = _args(16)
    got = ix_rsqrt(z)
    worst = 0.0
    with mp.workdps(50):
        for g, v in zip(got, z):
            ref = 1 / mp.sqrt(mp.mpf(float(v)))
            e = abs(mp.mpf(float(g)) - ref) / mp.mpf(float(np.spacing(float(ref))))
            worst = max(worst, float(e))
    assert worst < 0.52, worst


def test_rcp_rsqrt_special():
    """Exact cases and the arguments that go to the division / libm root."""
    z = np.array([1.0, 2.0, 4.0, 0.25, 2.0 ** -1022, 2.0 ** 1021])
    assert np.array_equal(ix_rcp(z), 1.0 / z)
    assert np.array_equal(ix_rsqrt(np.array([1.0, 4.0, 0.25, 2.0 ** 1022, 2.0 ** -1022])),
                          [1.0, 0.5, 2.0, 2.0 ** -511, 2.0 ** 511])
    odd = ix_rcp(np.array([0.0, -2.0, np.inf, 5e-324, 2.0 ** 1023]))
    assert odd[0] == np.inf and odd[1] == -0.5 and odd[2] == 0.0 and odd[4] == 2.0 ** -1023
    r = ix_rsqrt(np.array([0.0, -1.0, np.inf]))
    assert r[0] == np.inf and np.isnan(r[1]) and r[2] == 0.0


# --- fixed-point forms of the K-integral node chain ---------------------------

Q53 = Fraction(2) ** 53


def test_log_q53():
    """log z in Q53: within 0.56 units of 2^-53 of the exact logarithm (the
    polynomial stops at r^5: r^6/6 reaches 0.05 units in the first interval)
    (50-digit reference: near |log z| = 709 a unit of 2^-53 is 1.6e-19 of
    the value, finer than the double-double log resolves), over the whole normal range and at the
    reduction's interval edges; non-positive, subnormal and non-finite z give
    -2^62."""
    rng = np.random.default_rng(21)
    z = np.concatenate([np.exp(rng.uniform(-700, 700, 3000)), rng.uniform(1e-3, 200.0, 3000),
                        1.0 + np.arange(512) / 512.0, 1.0 + (np.arange(512) + 1) / 512.0 - 2.0 ** -52,
                        1.0 + np.arange(1, 50) * 2.0 ** -52, 2.0 - np.arange(1, 50) * 2.0 ** -52,
                        2.0 ** np.arange(-1022, 1023, 7), [2.2250738585072014e-308, 1.7976931348623157e308]])
    got = ix_log_q53(z)
    mp = pytest.importorskip("mpmath")
    with mp.workdps(50):
        for zi, g in zip(z, got):
            err = abs(mp.mpf(int(g)) - mp.log(mp.mpf(float(zi))) * 2 ** 53)
            assert err <= 0.56, (zi, int(g), float(err))
    odd = ix_log_q53(np.array([0.0, -1.0, 5e-324, np.inf, np.nan]))
    assert (odd == -(2 ** 62)).all()


def test_exp_q58_fx():
    """e^(d 2^-53) in Q58 from d in Q53: within 0.6 units of 2^-58 of the
    exact value; d chosen so that d 2^-53 is a double (the reference's
    argument), over [-42, 0] and at the reduction boundaries."""
    rng = np.random.default_rng(22)
    small = -rng.integers(0, 2 ** 53, 3000, dtype=np.int64)                       # |y| < 1, any bits
    big = -(rng.integers(0, 42 * 2 ** 47, 3000, dtype=np.int64) << 6)              # |y| < 42, 53 bits
    edges = np.array([-int(Fraction(np.log(2.0) / 512) * (k + Fraction(1, 2)) * Q53) // 64 * 64 for k in range(0, 800)],
                     dtype=np.int64)
    d = np.concatenate([small, big, edges, np.array([0, -1, -2 ** 40, -(41 * 2 ** 53)], dtype=np.int64)])
    got = ix_exp_q58_fx(d)
    scale = Fraction(2) ** 58
    for di, g in zip(d, got):
        y = Fraction(int(di)) / Q53
        assert Fraction(float(y)) == y
        hi, lo = oracle.dd_exp(float(y))
        exact = (Fraction(hi) + Fraction(lo)) * scale
        assert abs(Fraction(int(g)) - exact) <= Fraction(6, 10), (int(di), int(g), float(exact))
    assert int(ix_exp_q58_fx(np.array([0], dtype=np.int64))[0]) == 2 ** 58
    assert (ix_exp_q58_fx(np.array([-(42 * 2 ** 53), -(2 ** 62)], dtype=np.int64)) == 0).all()


def test_fix_and_mul_q58():
    """round(d 2^q) from the bit fields, and the Q58 x Q53 product, against
    exact rationals."""
    rng = np.random.default_rng(23)
    d = np.concatenate([rng.uniform(-16, 16, 2000), np.exp(rng.uniform(-60, 2.7, 1000)) * rng.choice([-1.0, 1.0], 1000),
                        [0.0, -0.0, 5e-324, 0.5, -0.5, 15.999999999999998, 2.0 ** -59, 3 * 2.0 ** -60]])
    for q in (53, 58):
        got = ix_fix(d, q)
        for di, g in zip(d, got):
            exact = Fraction(float(di)) * Fraction(2) ** q
            assert abs(Fraction(int(g)) - exact) <= Fraction(1, 2), (di, q, int(g))
    a = ix_fix(rng.uniform(-0.5, 16.0, 3000), 58)
    b = ix_fix(rng.uniform(-60.0, 60.0, 3000), 53)             # |a b| < 2^10
    got = ix_mul_q58(a, b)
    for ai, bi, g in zip(a, b, got):
        exact = Fraction(int(ai)) * Fraction(int(bi)) / Fraction(2) ** 58
        assert abs(Fraction(int(g)) - exact) <= Fraction(1, 2), (int(ai), int(bi), int(g))
