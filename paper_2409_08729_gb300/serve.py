"""Continuous-batching server over the C ABI (lb_server_* in include/logbessel.h).

Requests carry host arrays (submit) or CUDA tensors (submit_device, evaluated
in place); the native scheduler admits them as slots and device memory free
up, and a persistent kernel interleaves the work of all resident requests.
This module only marshals arguments.
"""
import ctypes

import numpy as np

from . import _binding as B

_KIND = {"i": 0, "k": 1}
_DT = {np.dtype(np.float64): B.LB_F64, np.dtype(np.float32): B.LB_F32}


class _Config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("idle_ms", ctypes.c_double)]


def _lib():
    L = B.lib()
    if not getattr(L, "_serve_ready", False):
        vp, i64, i32, ll = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_longlong
        L.lb_server_create.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(vp)]
        L.lb_server_submit.argtypes = [vp, i32, i32, vp, i64, vp, vp, i64, i32, ctypes.POINTER(ll)]
        L.lb_server_submit_device.argtypes = [vp, i32, i32, vp, i64, vp, vp, i64, i32, vp, ctypes.POINTER(ll)]
        L.lb_server_wait.argtypes = [vp, ll, ctypes.c_double]
        dp = ctypes.POINTER(ctypes.c_double)
        L.lb_server_ticket_info.argtypes = [vp, ll, ctypes.POINTER(i32), dp, dp, dp]
        L.lb_server_release.argtypes = [vp, ll]
        L.lb_server_stats.argtypes = [vp] + [ctypes.POINTER(ll)] * 4
        L.lb_server_device_stats.argtypes = [vp] + [ctypes.POINTER(ll)] * 3
        L.lb_server_destroy.argtypes = [vp]
        L.lb_server_last_error.argtypes = []
        L.lb_server_last_error.restype = ctypes.c_char_p
        for nm in ("lb_server_create", "lb_server_submit", "lb_server_submit_device", "lb_server_wait",
                   "lb_server_ticket_info",
                   "lb_server_release", "lb_server_stats", "lb_server_device_stats", "lb_server_destroy"):
            getattr(L, nm).restype = i32
        L._serve_ready = True
    return L


def _check(st):
    if st != B.LB_OK:
        raise B.LogBesselError(st, _lib().lb_server_last_error().decode())


class Server:
    def __init__(self, arena_bytes=1 << 30, max_slots=1024, ctas_per_sm=4, idle_ms=50.0):
        L = _lib()
        cfg = _Config(arena_bytes, max_slots, ctas_per_sm, idle_ms)
        h = ctypes.c_void_p()
        _check(L.lb_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, kind, v, x, out, mode="tight"):
        """Queue one request; v, x, out are host arrays (numpy or CPU torch
        tensors, pinned memory recommended).  v may hold a single order.
        Returns a ticket.  The arrays must stay alive until wait()."""
        arrs = []
        for a in (v, x, out):
            if hasattr(a, "data_ptr"):
                arrs.append((a.data_ptr(), np.dtype(str(a.dtype).replace("torch.", "")), a.numel(), a))
            else:
                a = np.ascontiguousarray(a)
                arrs.append((a.ctypes.data, a.dtype, a.size, a))
        (pv, dv, nv, ov), (px, dx, nx, ox), (po, do, no, oo) = arrs
        if not (dv == dx == do) or dx not in _DT:
            raise TypeError("v, x, out must share dtype float32 or float64")
        if no != nx or nv not in (1, nx):
            raise ValueError("shape mismatch")
        t = ctypes.c_longlong()
        _check(_lib().lb_server_submit(self._h, _KIND.get(kind, -1), _DT[dx], pv, 0 if nv == 1 else 1, px, po, nx,
                                       B.MODES.get(mode, -1), ctypes.byref(t)))
        self._keep[t.value] = (ov, ox, oo)
        return t.value

    def submit_device(self, kind, v, x, out, mode="tight", ready="stream"):
        """Queue one request on CUDA tensors of the server's device (v one
        order or one per pair, x and out contiguous, one dtype); the results
        are written to out in place.  `ready` says when the inputs are
        complete: "stream" (default) records an event on the current stream,
        so inputs written by work queued before the call are used; a
        torch.cuda.Event recorded after the writes; or None when they are
        complete already.  The tensors must stay alive until wait()."""
        import torch
        for a in (v, x, out):
            if not isinstance(a, torch.Tensor) or a.device.type != "cuda" or not a.is_contiguous():
                raise ValueError("submit_device takes contiguous CUDA tensors")
        if not (v.dtype == x.dtype == out.dtype) or x.dtype not in (torch.float32, torch.float64):
            raise TypeError("v, x, out must share dtype float32 or float64")
        if out.numel() != x.numel() or v.numel() not in (1, x.numel()):
            raise ValueError("shape mismatch")
        if isinstance(ready, str):
            ready = torch.cuda.Event()
            ready.record(torch.cuda.current_stream(x.device))
        code = B.LB_F64 if x.dtype == torch.float64 else B.LB_F32
        t = ctypes.c_longlong()
        _check(_lib().lb_server_submit_device(self._h, _KIND.get(kind, -1), code, v.data_ptr(),
                                              0 if v.numel() == 1 else 1, x.data_ptr(), out.data_ptr(),
                                              x.numel(), B.MODES.get(mode, -1),
                                              ctypes.c_void_p(ready.cuda_event if ready is not None else None),
                                              ctypes.byref(t)))
        self._keep[t.value] = (v, x, out, ready)
        return t.value

    def submit_ptr(self, kind, dtype, v, v_stride, x, out, n, device=False, mode="tight"):
        """Queue one request given raw pointers (ints): kind 'i' or 'k',
        dtype LB_F64 or LB_F32, v_stride 0 or 1; host pointers, or device
        pointers with device=True (inputs complete now).  For callers that
        keep their buffers alive themselves and submit at high rates: no
        argument inspection, no references kept."""
        t = ctypes.c_longlong()
        L = _lib()
        if device:
            st = L.lb_server_submit_device(self._h, _KIND[kind], dtype, v, v_stride, x, out, n, B.MODES[mode], None,
                                           ctypes.byref(t))
        else:
            st = L.lb_server_submit(self._h, _KIND[kind], dtype, v, v_stride, x, out, n, B.MODES[mode],
                                    ctypes.byref(t))
        if st != B.LB_OK:
            _check(st)
        return t.value

    def wait(self, ticket, timeout=60.0):
        _check(_lib().lb_server_wait(self._h, ticket, float(timeout)))
        self._keep.pop(ticket, None)

    def info(self, ticket):
        done = ctypes.c_int()
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(_lib().lb_server_ticket_info(self._h, ticket, ctypes.byref(done), ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)))
        return bool(done.value), a.value, b.value, c.value

    def release(self, ticket):
        _check(_lib().lb_server_release(self._h, ticket))

    def stats(self):
        v = [ctypes.c_longlong() for _ in range(4)]
        _check(_lib().lb_server_stats(self._h, *[ctypes.byref(a) for a in v]))
        return dict(zip(("completed", "evals", "kernel_launches", "in_flight"), [a.value for a in v]))

    FAMILIES = ("tiles_i_f64", "tiles_k_f64", "tiles_i_f32", "tiles_k_f32", "kint_f64_c0", "kint_f64_c1",
                "kint_f64_c2", "kint_f64_c3", "kint_f64_c4", "kint_f64_c5", "kint_f32")

    def device_stats(self):
        """The persistent kernel's device time accounts, cumulative: claim_ns
        (claiming and waiting for items, summed over CTAs), and per item
        family the summed busy ns and the items run."""
        nf = len(self.FAMILIES)
        claim = ctypes.c_longlong()
        busy = (ctypes.c_longlong * nf)()
        items = (ctypes.c_longlong * nf)()
        _check(_lib().lb_server_device_stats(self._h, ctypes.byref(claim), busy, items))
        return {"claim_ns": claim.value, "busy_ns": dict(zip(self.FAMILIES, list(busy))),
                "items": dict(zip(self.FAMILIES, list(items)))}

    def close(self):
        if self._h:
            _lib().lb_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
