"""Host build of the integer-pipe exp and log (csrc/lb_intmath.cuh).

The functions are integer code plus two single-precision operations, so a
host compilation gives the same bits as the GPU; the tests use it to check
them on the CPU and to compare the GPU results bit for bit."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2409_08729_gb300", "csrc")
_SRC = r'''
#include "lb_intmath.cuh"
extern "C" void ix_exp_arr(const double* y, double* o, long n) { for (long i = 0; i < n; ++i) o[i] = lb::ix_exp(y[i]); }
extern "C" void ix_log_arr(const double* y, double* o, long n) { for (long i = 0; i < n; ++i) o[i] = lb::ix_log(y[i]); }
extern "C" void ix_rcp_arr(const double* y, double* o, long n) { for (long i = 0; i < n; ++i) o[i] = lb::ix_rcp(y[i]); }
extern "C" void ix_rsqrt_arr(const double* y, double* o, long n) { for (long i = 0; i < n; ++i) o[i] = lb::ix_rsqrt(y[i]); }
extern "C" void ix_exp_q58_arr(const double* y, unsigned long long* o, long n) {
  for (long i = 0; i < n; ++i) o[i] = lb::ix_exp_q58(y[i]);
}
extern "C" void ix_log_q53_arr(const double* z, long long* o, long n) {
  for (long i = 0; i < n; ++i) o[i] = lb::ix_log_q53(z[i]);
}
extern "C" void ix_exp_q58_fx_arr(const long long* d, unsigned long long* o, long n) {
  for (long i = 0; i < n; ++i) o[i] = lb::ix_exp_q58_fx(d[i]);
}
extern "C" void ix_fix_arr(const double* d, int q, long long* o, long n) {
  for (long i = 0; i < n; ++i) o[i] = lb::ix_fix(d[i], q);
}
extern "C" void ix_mul_q58_arr(const long long* a, const long long* b, long long* o, long n) {
  for (long i = 0; i < n; ++i) o[i] = lb::ix_mul_q58(a[i], b[i]);
}
'''
_lib = None


def lib():
    global _lib
    if _lib is None:
        d = tempfile.mkdtemp(prefix="lb_intmath_")
        src = os.path.join(d, "ix.cpp")
        so = os.path.join(d, "ix.so")
        with open(src, "w") as f:
            f.write(_SRC)
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, "-o", so, src],
                       check=True)
        _lib = ctypes.CDLL(so)
    return _lib


def _run(name, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    o = np.empty_like(a)
    getattr(lib(), name)(a.ctypes.data_as(ctypes.c_void_p), o.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(a.size))
    return o


def ix_exp(a):
    return _run("ix_exp_arr", a)


def ix_log(a):
    return _run("ix_log_arr", a)


def ix_exp_q58(a):
    """e^a in Q58 fixed point (uint64)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    o = np.empty(a.size, dtype=np.uint64)
    lib().ix_exp_q58_arr(a.ctypes.data_as(ctypes.c_void_p), o.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(a.size))
    return o


def ix_rcp(a):
    return _run("ix_rcp_arr", a)


def ix_rsqrt(a):
    return _run("ix_rsqrt_arr", a)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def ix_log_q53(z):
    """log z in Q53 (int64)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    o = np.empty(z.size, dtype=np.int64)
    lib().ix_log_q53_arr(_ptr(z), _ptr(o), ctypes.c_long(z.size))
    return o


def ix_exp_q58_fx(d):
    """e^(d 2^-53) in Q58 (uint64) for d <= 0 in Q53 (int64)."""
    d = np.ascontiguousarray(d, dtype=np.int64)
    o = np.empty(d.size, dtype=np.uint64)
    lib().ix_exp_q58_fx_arr(_ptr(d), _ptr(o), ctypes.c_long(d.size))
    return o


def ix_fix(d, q):
    """round(d 2^q) as int64."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    o = np.empty(d.size, dtype=np.int64)
    lib().ix_fix_arr(_ptr(d), ctypes.c_int(q), _ptr(o), ctypes.c_long(d.size))
    return o


def ix_mul_q58(a, b):
    """round(a b 2^-58) for int64 a (Q58) and b (Q53)."""
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    o = np.empty(a.size, dtype=np.int64)
    lib().ix_mul_q58_arr(_ptr(a), _ptr(b), _ptr(o), ctypes.c_long(a.size))
    return o
