"""Double-float arithmetic (csrc/lb_df.cuh), host build, against exact
rational arithmetic: conversions within 2^-47, the Horner step within a few
2^-48 of its terms, and the double-float Debye polynomials (debye_uk.h)
within 2^-45 of their absolute coefficient sums."""
import ctypes
import os
import subprocess
import sys
import tempfile
from fractions import Fraction

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2409_08729_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_debye  # noqa: E402

_SRC = r'''
#define __host__
#define __device__
#define __forceinline__ inline
#define __constant__
#include <math.h>
template <typename T> inline T lb_fma(T a, T b, T c);
template <> inline double lb_fma<double>(double a, double b, double c) { return fma(a, b, c); }
template <> inline float lb_fma<float>(float a, float b, float c) { return fmaf(a, b, c); }
#include "lb_df.cuh"
#include "debye_uk.h"
using lb::dfloat;
extern "C" void df_conv(const double* d, float* h, float* l, double* back, long n) {
  for (long i = 0; i < n; ++i) {
    dfloat a = lb::df_from_double(d[i]);
    h[i] = a.h; l[i] = a.l; back[i] = lb::df_to_double(a);
  }
}
extern "C" void df_mad(const float* in, float* out, long n) {   // (ah, al, th, tl, ch, cl) -> (h, l)
  for (long i = 0; i < n; ++i) {
    const float* q = in + 6 * i;
    dfloat r = lb::df_mul_add(lb::df_make(q[0], q[1]), lb::df_make(q[2], q[3]), lb::df_make(q[4], q[5]));
    out[2 * i] = r.h; out[2 * i + 1] = r.l;
  }
}
extern "C" void df_mul_add2(const float* in, float* out, long n) {   // mul and add of (a, b)
  for (long i = 0; i < n; ++i) {
    const float* q = in + 4 * i;
    dfloat m = lb::df_mul(lb::df_make(q[0], q[1]), lb::df_make(q[2], q[3]));
    dfloat s = lb::df_add(lb::df_make(q[0], q[1]), lb::df_make(q[2], q[3]));
    out[4 * i] = m.h; out[4 * i + 1] = m.l; out[4 * i + 2] = s.h; out[4 * i + 3] = s.l;
  }
}
// the Horner loop of debye_P_df (lb_expr.cuh) over the generated table
static dfloat P(int k, dfloat p) {
  const float(*c)[2] = lb_debye_df + lb_debye_df_off[k];
  dfloat r = lb::df_make(c[k][0], c[k][1]);
  for (int i = k - 1; i >= 0; --i) r = lb::df_mul_add(r, p, lb::df_make(c[i][0], c[i][1]));
  return r;
}
extern "C" void df_debye(int k, const double* p, double* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = lb::df_to_double(P(k, lb::df_from_double(p[i])));
}
// the same loop over the Q_k table (debye_Q_df)
static dfloat Q(int k, dfloat p) {
  const float(*c)[2] = lb_debye_qdf + lb_debye_df_off[k];
  dfloat r = lb::df_make(c[k][0], c[k][1]);
  for (int i = k - 1; i >= 0; --i) r = lb::df_mul_add(r, p, lb::df_make(c[i][0], c[i][1]));
  return r;
}
extern "C" void df_debye_q(int k, const double* p, double* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = lb::df_to_double(Q(k, lb::df_from_double(p[i])));
}
'''
_lib = None


def lib():
    global _lib
    if _lib is None:
        d = tempfile.mkdtemp(prefix="lb_df_")
        src, so = os.path.join(d, "df.cpp"), os.path.join(d, "df.so")
        with open(src, "w") as f:
            f.write(_SRC)
        # no contraction: the host evaluates the same single-precision
        # operations as the device (whose fused multiply-adds are explicit)
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, "-o", so, src],
                       check=True)
        _lib = ctypes.CDLL(so)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _frac(a):
    return Fraction(float(a))


def test_conversions():
    rng = np.random.default_rng(1)
    d = np.concatenate([np.exp(rng.uniform(np.log(2.0 ** -70), np.log(2.0 ** 70), 4000)) * rng.choice([-1, 1], 4000),
                        [1.0, -1.0, 0.1, 1.0 / 3.0, np.pi, 2.0 ** -74, 2.0 ** 99]])
    h, l, back = np.empty(d.size, np.float32), np.empty(d.size, np.float32), np.empty_like(d)
    lib().df_conv(_p(d), _p(h), _p(l), _p(back), ctypes.c_long(d.size))
    for di, hi, li, bi in zip(d, h, l, back):
        exact = Fraction(float(di))
        assert abs(_frac(hi) + _frac(li) - exact) <= abs(exact) * Fraction(1, 2 ** 47)
        assert abs(_frac(li)) <= abs(_frac(hi)) * Fraction(1, 2 ** 23)       # normalized pair
        assert abs(Fraction(float(bi)) - exact) <= abs(exact) * Fraction(1, 2 ** 47)
    # below 2^-126 the pair is zero; between 2^-126 and 2^-74 the low part is dropped
    tiny = np.array([1e-40, -1e-300, 0.0, 2.0 ** -100])
    h, l, back = np.empty(4, np.float32), np.empty(4, np.float32), np.empty(4)
    lib().df_conv(_p(tiny), _p(h), _p(l), _p(back), ctypes.c_long(4))
    assert list(h[:3]) == [0.0, 0.0, 0.0] and list(l) == [0.0] * 4 and h[3] == np.float32(2.0 ** -100)


def _rand_df(rng, n, lo=-20, hi=20):
    d = np.exp(rng.uniform(lo * np.log(2), hi * np.log(2), n)) * rng.choice([-1, 1], n)
    h = d.astype(np.float32)
    l = (d - h.astype(np.float64)).astype(np.float32)
    return h, l


def test_mul_add_step():
    rng = np.random.default_rng(2)
    n = 3000
    cols = []
    for _ in range(3):
        cols += list(_rand_df(rng, n))
    q = np.stack(cols, axis=1).astype(np.float32)        # ah al th tl ch cl
    # some additions with cancellation: c near -(a t), as a normalized pair
    for i in range(n // 4):
        at = -((_frac(q[i, 0]) + _frac(q[i, 1])) * (_frac(q[i, 2]) + _frac(q[i, 3])))
        q[i, 4] = np.float32(float(at))
        q[i, 5] = np.float32(float(at - _frac(q[i, 4])) * (1 + 1e-3 * rng.standard_normal()))
    out = np.empty((n, 2), np.float32)
    lib().df_mad(_p(np.ascontiguousarray(q)), _p(out), ctypes.c_long(n))
    for r, o in zip(q, out):
        a = _frac(r[0]) + _frac(r[1])
        t = _frac(r[2]) + _frac(r[3])
        c = _frac(r[4]) + _frac(r[5])
        exact = a * t + c
        bound = (abs(a * t) + abs(c)) * Fraction(6, 2 ** 48)
        assert abs(_frac(o[0]) + _frac(o[1]) - exact) <= bound, (r, o)


def test_mul_and_add():
    rng = np.random.default_rng(3)
    n = 3000
    q = np.stack(list(_rand_df(rng, n)) + list(_rand_df(rng, n)), axis=1).astype(np.float32)
    out = np.empty((n, 4), np.float32)
    lib().df_mul_add2(_p(np.ascontiguousarray(q)), _p(out), ctypes.c_long(n))
    for r, o in zip(q, out):
        a, b = _frac(r[0]) + _frac(r[1]), _frac(r[2]) + _frac(r[3])
        assert abs(_frac(o[0]) + _frac(o[1]) - a * b) <= abs(a * b) * Fraction(4, 2 ** 48)
        assert abs(_frac(o[2]) + _frac(o[3]) - (a + b)) <= (abs(a) + abs(b)) * Fraction(4, 2 ** 48)


@pytest.mark.parametrize("which", ["P", "Q"])
@pytest.mark.parametrize("k", [2, 5, 9, 13])
def test_debye_polynomials_in_double_float(k, which):
    """P_k(p) and Q_k(p) = k P_k + 2 p P_k' (the derivative's polynomials) in
    double-float against the exact rational polynomial at the double-float
    input; the error bound scales with sum |c_i| p^i, the size of the terms
    that cancel near p = 1."""
    cs = gen_debye.p_coeffs(k) if which == "P" else gen_debye.q_coeffs(k)
    p = np.concatenate([np.linspace(0.0, 1.0, 101), np.random.default_rng(k).uniform(0, 1, 200)])
    out = np.empty_like(p)
    getattr(lib(), "df_debye" if which == "P" else "df_debye_q")(ctypes.c_int(k), _p(p), _p(out), ctypes.c_long(p.size))
    h, l, back = np.empty(p.size, np.float32), np.empty(p.size, np.float32), np.empty_like(p)
    lib().df_conv(_p(p), _p(h), _p(l), _p(back), ctypes.c_long(p.size))
    for pi, hi, li, oi in zip(p, h, l, out):
        x = _frac(hi) + _frac(li)
        exact = sum(c * x ** i for i, c in enumerate(cs))
        scale = sum(abs(c) * x ** i for i, c in enumerate(cs))
        assert abs(Fraction(float(oi)) - exact) <= scale * Fraction(1, 2 ** 45) + abs(exact) * Fraction(1, 2 ** 52), (k, pi)
