"""ctypes binding of liblogbessel.so (argument marshalling only)."""
import ctypes
import os

from .build import LIB_PATH

LB_OK, LB_EINVAL, LB_ECUDA, LB_ENOMEM, LB_ETIMEOUT, LB_ENOTSUP = range(6)
LB_F64, LB_F32 = 0, 1
MODES = {"tight": 0, "paper_gpu": 1, "paper_cpu_order": 2}
REGIONS = {"mu20": 0, "u13": 1, "fallback": 2, "special": 3, "mu3": 4, "u4": 5, "u6": 6, "u9": 7}
STATUS_NAMES = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ECUDA", 3: "LB_ENOMEM", 4: "LB_ETIMEOUT", 5: "LB_ENOTSUP"}


class LogBesselError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load the library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblogbessel.so is not built (%s); run "
                              "paper_2409_08729_gb300.build.build_library()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        for name in ("logbessel_i", "logbessel_k", "logbessel_i_dx", "logbessel_k_dx"):
            f = getattr(L, name)
            f.argtypes = [i32, vp, i64, vp, vp, i64, i32, vp]
            f.restype = i32
        L.logbessel_workspace_bytes.argtypes = [i64]
        L.logbessel_workspace_bytes.restype = i64
        for name in ("logbessel_k_ws", "logbessel_k_dx_ws"):
            f = getattr(L, name)
            f.argtypes = [i32, vp, i64, vp, vp, i64, i32, vp, i64, vp]
            f.restype = i32
        L.logbessel_host.argtypes = [i32, i32, vp, i64, vp, vp, i64, i32, i64]
        L.logbessel_host.restype = i32
        L.logbessel_host_release.argtypes = []
        L.logbessel_host_release.restype = i32
        L.logbessel_vmf_log_c.argtypes = [i32, ctypes.c_double, vp, vp, i64, i32, vp]
        L.logbessel_vmf_log_c.restype = i32
        L.logbessel_classify.argtypes = [i32, i32, vp, i64, vp, vp, i64, i32, vp]
        L.logbessel_classify.restype = i32
        L.logbessel_eval_region.argtypes = [i32, i32, vp, i64, vp, vp, i64, i32, i32, vp]
        L.logbessel_eval_region.restype = i32
        L.logbessel_last_error.argtypes = []
        L.logbessel_last_error.restype = ctypes.c_char_p
        L.logbessel_version.argtypes = []
        L.logbessel_version.restype = ctypes.c_char_p
        L.logbessel_profile_enable.argtypes = [i32]
        L.logbessel_profile_enable.restype = None
        L.logbessel_profile_slots.argtypes = []
        L.logbessel_profile_slots.restype = i32
        L.logbessel_profile_get.argtypes = [i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                            ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
        L.logbessel_profile_get.restype = i32
        L.logbessel_measure_fp64.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
        L.logbessel_measure_fp64.restype = i32
        L.logbessel_math_eval.argtypes = [i32, vp, vp, i64, vp]
        L.logbessel_math_eval.restype = i32
        L.logbessel_launch_count.argtypes = []
        L.logbessel_launch_count.restype = ctypes.c_longlong
        _lib = L
    return _lib


def check(status):
    if status != LB_OK:
        raise LogBesselError(status, lib().logbessel_last_error().decode())
    return status


def profile_enable(on=True):
    lib().logbessel_profile_enable(1 if on else 0)


def profile_read():
    """{kernel name: (launches, timed launches, total ms)}; waits for timed launches."""
    out = {}
    for slot in range(lib().logbessel_profile_slots()):
        name = ctypes.c_char_p()
        la, tl, ms = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
        check(lib().logbessel_profile_get(slot, ctypes.byref(name), ctypes.byref(la), ctypes.byref(tl), ctypes.byref(ms)))
        out[name.value.decode()] = (la.value, tl.value, ms.value)
    return out


def launch_count():
    return lib().logbessel_launch_count()


def measure_fp64(stream=None):
    """Measured FP64 rates of the current GPU: {'dfma','exp','log','div','sqrt','lgamma'} per second."""
    rates = (ctypes.c_double * 13)()
    check(lib().logbessel_measure_fp64(rates, stream))
    return dict(zip(("dfma", "exp", "log", "div", "sqrt", "lgamma", "fm_exp", "fm_log", "fm_exp_term", "ix_exp", "ix_log",
                     "ix_rcp", "ix_rsqrt"), list(rates)))
