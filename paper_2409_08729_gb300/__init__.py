"""GB300 log-Bessel library: batched log I_v(x) and log K_v(x) on CUDA tensors.

Thin PyTorch-facing layer over the C ABI in include/logbessel.h.  Every step
of the evaluation runs in the library's CUDA kernels; this module only
broadcasts and allocates tensors and passes device pointers and the current
stream.  There is no CPU path: calls on CPU tensors raise.

Paper: Plesner, Sorensen, Hauberg, "Accurate Computation of the Logarithm of
Modified Bessel Functions on GPUs", ICS 2024 (arXiv 2409.08729).
"""
import torch

from . import _binding
from ._binding import LogBesselError, MODES, REGIONS
from .build import build_library

__all__ = ["log_i", "log_k", "log_i_dx", "log_k_dx", "host_eval", "classify", "eval_region", "LogBesselError", "MODES", "REGIONS",
           "build_library", "version"]


def version():
    return _binding.lib().logbessel_version().decode()


def _dtype_code(dt):
    if dt == torch.float64:
        return _binding.LB_F64
    if dt == torch.float32:
        return _binding.LB_F32
    raise TypeError("log-Bessel functions take float64 or float32 tensors, got %s" % dt)


def _prep(v, x):
    """Broadcast (v, x) to CUDA tensors of a common float dtype.

    Returns (v_flat, v_stride, x_flat, shape).  A scalar order is passed with
    stride 0 instead of being expanded."""
    if not isinstance(x, torch.Tensor):
        raise TypeError("x must be a CUDA tensor")
    if x.device.type != "cuda":
        raise ValueError("x must be on a CUDA device (the library has no CPU path)")
    dt = x.dtype if x.dtype in (torch.float32, torch.float64) else torch.float64
    if not isinstance(v, torch.Tensor):
        v = torch.tensor(float(v), dtype=dt, device=x.device)
    if v.device != x.device:
        raise ValueError("v and x must be on the same device")
    v = v.to(dt)
    x = x.to(dt)
    if v.numel() == 1:
        shape = x.shape
        return v.reshape(1).contiguous(), 0, x.contiguous().reshape(-1), shape
    vb, xb = torch.broadcast_tensors(v, x)
    shape = xb.shape
    return vb.contiguous().reshape(-1), 1, xb.contiguous().reshape(-1), shape


def _stream(dev):
    return ctypes_stream(torch.cuda.current_stream(dev))


def ctypes_stream(s):
    return s.cuda_stream


def _call(name, v, x, mode, out):
    vf, vs, xf, shape = _prep(v, x)
    n = xf.numel()
    if out is None:
        out = torch.empty(shape, dtype=xf.dtype, device=xf.device)
    elif out.shape != shape or out.dtype != xf.dtype or not out.is_contiguous():
        raise ValueError("out must be a contiguous %s tensor of shape %s" % (xf.dtype, tuple(shape)))
    with torch.cuda.device(xf.device):
        fn = getattr(_binding.lib(), name)
        _binding.check(fn(_dtype_code(xf.dtype), vf.data_ptr(), vs, xf.data_ptr(), out.data_ptr(), n,
                          MODES[mode], _stream(xf.device)))
    return out


class _LogBesselFn(torch.autograd.Function):
    """Forward log I or log K; backward multiplies by the hand-written adjoint
    kernel (d/dx log I_v = I'_v/I_v, d/dx log K_v = K'_v/K_v).  The gradient
    with respect to the order v is not provided."""

    @staticmethod
    def forward(ctx, v, x, kind, mode):
        ctx.save_for_backward(v, x)
        ctx.kind, ctx.mode = kind, mode
        return _call("logbessel_i" if kind == "i" else "logbessel_k", v, x, mode, None)

    @staticmethod
    def backward(ctx, grad):
        v, x = ctx.saved_tensors
        if ctx.needs_input_grad[0]:
            raise NotImplementedError("the derivative with respect to the order v is not provided")
        d = _call("logbessel_i_dx" if ctx.kind == "i" else "logbessel_k_dx", v, x, ctx.mode, None)
        gx = grad * d
        if gx.shape != x.shape:
            gx = gx.sum_to_size(x.shape)
        return None, gx, None, None


def _with_grad(kind, v, x, mode, out):
    if out is None and isinstance(x, torch.Tensor) and x.requires_grad and torch.is_grad_enabled():
        if not isinstance(v, torch.Tensor):
            v = torch.tensor(float(v), dtype=x.dtype, device=x.device)
        return _LogBesselFn.apply(v, x, kind, mode)
    return _call("logbessel_i" if kind == "i" else "logbessel_k", v, x, mode, out)


def log_i(v, x, mode="tight", out=None):
    """log I_v(x) elementwise (v >= 0, x >= 0); v broadcasts against x.
    Differentiable in x (autograd uses the adjoint kernel)."""
    return _with_grad("i", v, x, mode, out)


def log_k(v, x, mode="tight", out=None):
    """log K_v(x) elementwise (real v, x >= 0); v broadcasts against x.
    Differentiable in x (autograd uses the adjoint kernel)."""
    return _with_grad("k", v, x, mode, out)


def log_i_dx(v, x, mode="tight", out=None):
    """d/dx log I_v(x) = I'_v(x)/I_v(x) elementwise."""
    return _call("logbessel_i_dx", v, x, mode, out)


def log_k_dx(v, x, mode="tight", out=None):
    """d/dx log K_v(x) = K'_v(x)/K_v(x) elementwise."""
    return _call("logbessel_k_dx", v, x, mode, out)


_HOST_FN = {"log_i": 0, "log_k": 1, "log_i_dx": 2, "log_k_dx": 3}


def host_eval(fn, v, x, out=None, mode="tight", chunk=0):
    """End-to-end evaluation on host arrays (numpy, or CPU tensors; pinned
    memory overlaps the copies with the computation).  fn is 'log_i',
    'log_k', 'log_i_dx' or 'log_k_dx'; v is one order or an array like x."""
    import numpy as np
    if isinstance(x, torch.Tensor):
        xa = x
        dt = x.dtype
        n = x.numel()
        xp = x.data_ptr()
        va = v if isinstance(v, torch.Tensor) else torch.tensor([float(v)], dtype=dt)
        vp, vs = va.data_ptr(), (0 if va.numel() == 1 else 1)
        if out is None:
            out = torch.empty_like(x)
        op = out.data_ptr()
        code = _dtype_code(dt)
        keep = (xa, va, out)
    else:
        xa = np.ascontiguousarray(x)
        if xa.dtype not in (np.float32, np.float64):
            xa = xa.astype(np.float64)
        va = np.ascontiguousarray(np.atleast_1d(np.asarray(v, dtype=xa.dtype)))
        if out is None:
            out = np.empty_like(xa)
        n, xp, vp, op = xa.size, xa.ctypes.data, va.ctypes.data, out.ctypes.data
        vs = 0 if va.size == 1 else 1
        code = _binding.LB_F64 if xa.dtype == np.float64 else _binding.LB_F32
        keep = (xa, va, out)
    _binding.check(_binding.lib().logbessel_host(_HOST_FN[fn], code, vp, vs, xp, op, n, MODES[mode], int(chunk)))
    del keep
    return out


def host_release():
    """Free the device buffer, streams and events that host_eval keeps for
    the current device between calls."""
    _binding.check(_binding.lib().logbessel_host_release())


def classify(kind, v, x, mode="tight"):
    """Region id (uint8, see REGIONS) of every pair; kind is 'i' or 'k'."""
    vf, vs, xf, shape = _prep(v, x)
    out = torch.empty(shape, dtype=torch.uint8, device=xf.device)
    with torch.cuda.device(xf.device):
        _binding.check(_binding.lib().logbessel_classify(0 if kind == "i" else 1, _dtype_code(xf.dtype),
                                                         vf.data_ptr(), vs, xf.data_ptr(), out.data_ptr(),
                                                         xf.numel(), MODES[mode], _stream(xf.device)))
    return out


def eval_region(kind, region, v, x, mode="tight"):
    """Evaluate one expression (a REGIONS name) for every pair, without dispatch."""
    vf, vs, xf, shape = _prep(v, x)
    out = torch.empty(shape, dtype=xf.dtype, device=xf.device)
    with torch.cuda.device(xf.device):
        _binding.check(_binding.lib().logbessel_eval_region(0 if kind == "i" else 1, _dtype_code(xf.dtype),
                                                            vf.data_ptr(), vs, xf.data_ptr(), out.data_ptr(),
                                                            xf.numel(), REGIONS[region], MODES[mode],
                                                            _stream(xf.device)))
    return out
