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
