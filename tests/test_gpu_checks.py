"""The checked build (liblogbessel_checks.so, compiled with LB_CHECKS).

There every index into a tile's shared list, into the K-integral queue, and
every pair offset read back from the queue is checked against its bound;
a failed check sets a bit of a device status word instead of touching memory
out of range.  The path runs here over ragged sizes around the tile and warp
widths, every region and rule class, mixed and single orders, the paper's
dispatches, the derivatives, a caller workspace small enough to force many
passes and the entry point without allocation; the status word must stay
clear, and every result must equal the release build's bit for bit (the
checks only read)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_08729_gb300 import _binding as B
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = (1, 31, 33, 1023, 1024, 1025, 4097, 65537, 300001)


def _declare(L):
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    for name in ("logbessel_i", "logbessel_k", "logbessel_i_dx", "logbessel_k_dx", "logbessel_k_noalloc"):
        f = getattr(L, name)
        f.argtypes = [i32, vp, i64, vp, vp, i64, i32, vp]
        f.restype = i32
    L.logbessel_k_ws.argtypes = [i32, vp, i64, vp, vp, i64, i32, vp, i64, vp]
    L.logbessel_k_ws.restype = i32
    L.logbessel_check_status.argtypes = [ctypes.POINTER(ctypes.c_uint), i32]
    L.logbessel_check_status.restype = i32
    return L


@pytest.fixture(scope="module")
def libs(cuda):
    from paper_2409_08729_gb300.build import CHECKS_LIB_PATH, build_library
    build_library()
    return _declare(B.lib()), _declare(ctypes.CDLL(CHECKS_LIB_PATH))


def _status(L):
    bits = ctypes.c_uint(0)
    st = L.logbessel_check_status(ctypes.byref(bits), 1)
    return st, bits.value


def _pairs(n, seed):
    """A mix over the whole domain with a third of the pairs in the K
    integral (every rule class) and some domain edges."""
    rng = np.random.default_rng(seed)
    v, x = W.robust_pairs(n, seed=seed, vmax=1e4, xmin=1e-6, xmax=1e4)
    k = n // 3
    v[:k] = rng.choice([0.0, 0.05, 0.3, 0.6, 1.0, 2.5, 4.0, 9.0, 16.0], k)
    x[:k] = np.exp(rng.uniform(np.log(1e-300), np.log(25.0), k))
    ev, ex = W.edge_pairs()
    m = min(n, ev.size) // 2
    if m:
        v[-m:], x[-m:] = ev[:m], ex[:m]
    p = rng.permutation(n)
    return v[p], x[p]


def _run(L, fn, dt, v, vs, x, n, mode=0, extra=()):
    out = torch.full_like(x, float("nan"))
    st = getattr(L, fn)(dt, v.data_ptr(), vs, x.data_ptr(), out.data_ptr(), n, mode, *extra)
    assert st == B.LB_OK, (fn, st, L.logbessel_last_error())
    return out


def _same(a, b):
    return torch.equal(a.view(torch.int64) if a.dtype == torch.float64 else a.view(torch.int32),
                       b.view(torch.int64) if b.dtype == torch.float64 else b.view(torch.int32))


def test_release_build_reports_no_checks(libs):
    R, _ = libs
    st, bits = _status(R)
    assert st == B.LB_ENOTSUP and bits == 0


def test_checked_build_matches_release_and_stays_clear(libs, cuda):
    R, C = libs
    assert _status(C) == (B.LB_OK, 0)
    stream = torch.cuda.current_stream(cuda).cuda_stream
    cases = 0
    for n in SIZES:
        v, x = _pairs(n, seed=n)
        for dt, tdt in ((B.LB_F64, torch.float64), (B.LB_F32, torch.float32)):
            tv, tx = torch.tensor(v, dtype=tdt, device=cuda), torch.tensor(x, dtype=tdt, device=cuda)
            fns = ("logbessel_i", "logbessel_k") + (("logbessel_i_dx", "logbessel_k_dx") if dt == B.LB_F64 else ())
            for fn in fns:
                a = _run(R, fn, dt, tv, 1, tx, n, extra=(stream,))
                b = _run(C, fn, dt, tv, 1, tx, n, extra=(stream,))
                assert _same(a, b), (fn, n, dt)
                cases += 1
            for order in (0.0, 0.6, 3.0, 12.0, 100.0):          # one order for all pairs
                to = torch.tensor([order], dtype=tdt, device=cuda)
                for fn in ("logbessel_i", "logbessel_k"):
                    assert _same(_run(R, fn, dt, to, 0, tx, n, extra=(stream,)),
                                 _run(C, fn, dt, to, 0, tx, n, extra=(stream,))), (fn, n, order)
                    cases += 1
        tv, tx = torch.tensor(v, device=cuda), torch.tensor(x, device=cuda)
        for mode in (1, 2):                                      # the paper's dispatches
            for fn in ("logbessel_i", "logbessel_k"):
                assert _same(_run(R, fn, B.LB_F64, tv, 1, tx, n, mode, (stream,)),
                             _run(C, fn, B.LB_F64, tv, 1, tx, n, mode, (stream,))), (fn, n, mode)
                cases += 1
        # a caller workspace of 2048-pair passes, and the entry point without allocation
        ws = torch.empty(8448 // 8, dtype=torch.float64, device=cuda)
        assert _same(_run(R, "logbessel_k_ws", B.LB_F64, tv, 1, tx, n, 0, (ws.data_ptr(), 8448, stream)),
                     _run(C, "logbessel_k_ws", B.LB_F64, tv, 1, tx, n, 0, (ws.data_ptr(), 8448, stream)))
        assert _same(_run(R, "logbessel_k", B.LB_F64, tv, 1, tx, n, extra=(stream,)),
                     _run(C, "logbessel_k_noalloc", B.LB_F64, tv, 1, tx, n, extra=(stream,)))
        cases += 2
    torch.cuda.synchronize()
    st, bits = _status(C)
    assert st == B.LB_OK and bits == 0, bits
    assert cases > 200
