"""Extended-precision CPU oracle for log I_v(x), log K_v(x) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library itself never calls it; the
CUDA path has no CPU fallback.

The evaluator is plain C (``logbessel_oracle.c``) in double-double arithmetic:
log I_v(x) from the positive-term power series (paper Sec. 3.1, the infinite
series of I_v), log K_v(x) from the integral int_0^inf exp(-x cosh t) cosh(vt)
dt (DLMF 10.32.9) by the trapezoid rule.  Neither uses the paper's asymptotic
expansions or its Rothwell integral, so the two sides share no formula.
The same source also builds on the C type long double (binary128 on aarch64,
80-bit on x86-64) with libm's long double functions: ``log_i_ld``,
``log_k_ld``; its agreement with the double-double build pins the
double-double arithmetic layer.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "logbessel_oracle.c")
_SO = os.path.join(_HERE, "_build", "liblogbessel_oracle.so")
# the same evaluators compiled on the C type long double (binary128 on
# aarch64, 80-bit x87 on x86-64) instead of double-double
_SO_LD = os.path.join(_HERE, "_build", "liblogbessel_oracle_ld.so")

OP_LOG_I, OP_LOG_K, OP_DLOG_I, OP_DLOG_K, OP_DV_I, OP_DV_K, OP_VMF = range(7)

_lib = None


def _compile(so, defines):
    os.makedirs(os.path.dirname(so), exist_ok=True)
    if os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    tmp = so + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"] + defines + \
          [_SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, so)
    return so


def build(force=False):
    """Compile the oracle with gcc (no fast-math, no FMA contraction): the
    double-double build and the long double build of the same source."""
    if force:
        for so in (_SO, _SO_LD):
            if os.path.exists(so):
                os.remove(so)
    _compile(_SO_LD, ["-DORACLE_LONG_DOUBLE"])
    return _compile(_SO, [])


def _declare(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_eval.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int64, ctypes.c_int]
    lib.oracle_eval.restype = ctypes.c_int
    lib.oracle_significand_bits.argtypes = []
    lib.oracle_significand_bits.restype = ctypes.c_int
    return lib


_lib_ld = None


def _load_ld():
    global _lib_ld
    if _lib_ld is None:
        build()
        _lib_ld = _declare(ctypes.CDLL(_SO_LD))
    return _lib_ld


def _load():
    global _lib
    if _lib is None:
        lib = _declare(ctypes.CDLL(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_eval.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int64, ctypes.c_int]
        lib.oracle_eval.restype = ctypes.c_int
        for name in ("oracle_dd_exp", "oracle_dd_log", "oracle_dd_lgamma", "oracle_dd_log1p"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            f.restype = None
        lib.oracle_dd_const.argtypes = [ctypes.c_int, dp]
        lib.oracle_dd_const.restype = None
        _lib = lib
    return _lib


def default_threads():
    return os.cpu_count() or 1


def _eval(op, a, b, threads=None, want_lo=False, lib=None):
    lib = lib or _load()
    a, b = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64))
    shape = a.shape
    a = np.ascontiguousarray(a.ravel())
    b = np.ascontiguousarray(b.ravel())
    out = np.empty(a.size, dtype=np.float64)
    lo = np.empty(a.size, dtype=np.float64) if want_lo else None
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_eval(op, a.ctypes.data_as(dp), b.ctypes.data_as(dp), out.ctypes.data_as(dp),
                         lo.ctypes.data_as(dp) if want_lo else None, a.size,
                         threads or default_threads())
    if rc != 0:
        raise RuntimeError("oracle thread creation failed")
    if want_lo:
        return out.reshape(shape), lo.reshape(shape)
    return out.reshape(shape)


def log_i(v, x, threads=None, want_lo=False):
    """log I_v(x) (double, or (hi, lo) pair with want_lo)."""
    return _eval(OP_LOG_I, v, x, threads, want_lo)


def log_k(v, x, threads=None, want_lo=False):
    """log K_v(x) (double, or (hi, lo) pair with want_lo)."""
    return _eval(OP_LOG_K, v, x, threads, want_lo)


def long_double_bits():
    """Significand bits of the long double build: 113 (binary128, aarch64
    Linux) or 64 (x87 extended, x86-64)."""
    return _load_ld().oracle_significand_bits()


def log_i_ld(v, x, threads=None):
    """log I_v(x) from the long double build of the same evaluator, as a
    (hi, lo) pair of doubles (hi + lo carries the long double result)."""
    return _eval(OP_LOG_I, v, x, threads, True, _load_ld())


def log_k_ld(v, x, threads=None):
    """log K_v(x) from the long double build, as a (hi, lo) pair."""
    return _eval(OP_LOG_K, v, x, threads, True, _load_ld())


def dlog_i_dx(v, x, threads=None):
    """d/dx log I_v(x) = I_{v+1}(x)/I_v(x) + v/x."""
    return _eval(OP_DLOG_I, v, x, threads)


def dlog_k_dx(v, x, threads=None):
    """d/dx log K_v(x) = -(K_{v-1}(x)/K_v(x) + v/x)."""
    return _eval(OP_DLOG_K, v, x, threads)


def dlog_i_dv(v, x, threads=None):
    """d/dv log I_v(x) by a double-double central difference."""
    return _eval(OP_DV_I, v, x, threads)


def dlog_k_dv(v, x, threads=None):
    """d/dv log K_v(x) by a double-double central difference."""
    return _eval(OP_DV_K, v, x, threads)


def vmf_log_c(d, kappa, threads=None):
    """log C_d(kappa) = (d/2-1) log kappa - (d/2) log 2pi - log I_{d/2-1}(kappa)."""
    return _eval(OP_VMF, d, kappa, threads)


def dd_exp(hi, lo=0.0):
    out = (ctypes.c_double * 2)()
    _load().oracle_dd_exp(hi, lo, out)
    return out[0], out[1]


def dd_log(hi, lo=0.0):
    out = (ctypes.c_double * 2)()
    _load().oracle_dd_log(hi, lo, out)
    return out[0], out[1]


def dd_log1p(hi, lo=0.0):
    out = (ctypes.c_double * 2)()
    _load().oracle_dd_log1p(hi, lo, out)
    return out[0], out[1]


def dd_lgamma(hi, lo=0.0):
    out = (ctypes.c_double * 2)()
    _load().oracle_dd_lgamma(hi, lo, out)
    return out[0], out[1]


def dd_const(which):
    """0 -> ln 2, 1 -> pi, as (hi, lo)."""
    out = (ctypes.c_double * 2)()
    _load().oracle_dd_const(which, out)
    return out[0], out[1]


def error_scale(kind, v, x, threads=None):
    """Scale c = max(1, |x df/dx|, |v df/dv|) of the error metric
    err = |got - ref| / max(|ref|, c); f = log I (kind 'i') or log K ('k').

    An input perturbed by one rounding moves f by about eps * c, so no
    double-precision evaluation can beat that floor.
    """
    v = np.asarray(v, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if kind == "i":
        dx, dv = dlog_i_dx(v, x, threads), dlog_i_dv(v, x, threads)
    else:
        dx, dv = dlog_k_dx(v, x, threads), dlog_k_dv(v, x, threads)
    with np.errstate(invalid="ignore"):
        c = np.fmax(np.abs(x * dx), np.abs(v * dv))
    c = np.where(np.isfinite(c), c, 1.0)
    return np.maximum(c, 1.0)


def rel_err(got, ref, scale):
    """|got - ref| / max(|ref|, scale); exact matches of non-finite values give 0."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    with np.errstate(invalid="ignore", over="ignore"):
        e = np.abs(got - ref) / np.maximum(np.abs(ref), scale)
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    return np.where(same, 0.0, np.where(np.isnan(e), np.inf, e))
