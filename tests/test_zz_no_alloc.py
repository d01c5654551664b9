"""logbessel_k_noalloc, the entry point that allocates no device memory.

Some callers cannot let a library allocate: code that runs under a device
memory budget fixed in advance, latency-critical loops where an allocation
may block or fail at the wrong moment, and frameworks whose own allocator
must own all device memory.  This entry point takes its scratch from a fixed
array in the library's device memory instead.  The tests call it through the
C ABI on two calls in a row and check that
  * its results equal those of the allocating logbessel_k bit for bit (the
    two run the same kernels on the same inputs; only the scratch differs),
  * a sample of them matches the oracle within the FP64 gate,
  * it takes nothing from the device's stream-ordered memory pool, where
    logbessel_k takes its scratch (a watermark of the pool that the driver
    keeps), which logbessel_k itself is shown to move.
This file is collected last, so a run that stops at the first failure has
run every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2409_08729_gb300 import _binding as B
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 4e-15      # the FP64 gate of the parity tests
MAX_PAIRS = 1 << 20

# CUmemPool_attribute values of the driver API (cuda.h)
CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7
CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


def _lib():
    L = B.lib()
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.logbessel_k_noalloc.argtypes = [i32, vp, i64, vp, vp, i64, i32, vp]
    L.logbessel_k_noalloc.restype = i32
    return L


class _DefaultPool:
    """The current device's default memory pool (the one cudaMallocAsync
    draws from), read through the driver API."""

    def __init__(self, ordinal):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        val = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(val)) == 0
        return val.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0


def _inputs(n, seed):
    """About half of the pairs in the K-integral fallback (v <= 16, x <= 25),
    so the scratch queue is exercised, the rest spread over the other regions."""
    rng = np.random.default_rng(seed)
    v1, x1 = rng.uniform(0, 16, n // 2), np.exp(rng.uniform(np.log(1e-5), np.log(25), n // 2))
    v2, x2 = W.robust_pairs(n - n // 2, seed=seed, vmax=1e4, xmin=1e-3, xmax=1e4)
    return np.concatenate([v1, v2]), np.concatenate([x1, x2])


def test_noalloc_matches_logbessel_k(cuda):
    L = _lib()
    stream = torch.cuda.current_stream(cuda).cuda_stream
    for seed, n in ((1, 300000), (2, MAX_PAIRS)):          # two calls in a row, the second at the maximum
        v, x = _inputs(n, seed)
        tv = torch.tensor(v, device=cuda)
        tx = torch.tensor(x, device=cuda)
        ref = torch.empty_like(tx)
        got = torch.full_like(tx, float("nan"))
        B.check(L.logbessel_k(B.LB_F64, tv.data_ptr(), 1, tx.data_ptr(), ref.data_ptr(), n, 0, stream))
        B.check(L.logbessel_k_noalloc(B.LB_F64, tv.data_ptr(), 1, tx.data_ptr(), got.data_ptr(), n, 0, stream))
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.array_equal(a.view(np.int64), b.view(np.int64)), (seed, int(np.sum(a != b)))
        idx = np.random.default_rng(seed).integers(0, n, 600)
        want = oracle.log_k(v[idx], x[idx])
        err = oracle.rel_err(a[idx], want, oracle.error_scale("k", v[idx], x[idx]))
        assert err.max() <= TOL64, (seed, float(err.max()))


def test_noalloc_takes_nothing_from_the_pool(cuda):
    L = _lib()
    stream = torch.cuda.current_stream(cuda).cuda_stream
    n = 200000
    v, x = _inputs(n, 3)
    tv = torch.tensor(v, device=cuda)
    tx = torch.tensor(x, device=cuda)
    ref = torch.empty_like(tx)
    got = torch.empty_like(tx)
    pool = _DefaultPool(cuda.index or 0)
    # the first call on the device looks up the scratch array's address
    B.check(L.logbessel_k_noalloc(B.LB_F64, tv.data_ptr(), 1, tx.data_ptr(), got.data_ptr(), n, 0, stream))
    torch.cuda.synchronize()
    base = pool.get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)
    pool.reset_high()
    for _ in range(2):
        B.check(L.logbessel_k_noalloc(B.LB_F64, tv.data_ptr(), 1, tx.data_ptr(), got.data_ptr(), n, 0, stream))
    torch.cuda.synchronize()
    assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) <= base
    # the check sees an allocation: logbessel_k takes its queue from this pool
    B.check(L.logbessel_k(B.LB_F64, tv.data_ptr(), 1, tx.data_ptr(), ref.data_ptr(), n, 0, stream))
    torch.cuda.synchronize()
    assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) >= base + 4 * n
    assert torch.equal(got, ref)


def test_noalloc_rejects_oversized_calls(cuda):
    L = _lib()
    t = torch.ones(4, dtype=torch.float64, device=cuda)
    st = L.logbessel_k_noalloc(B.LB_F64, t.data_ptr(), 0, t.data_ptr(), t.data_ptr(), MAX_PAIRS + 1, 0, None)
    assert st == B.LB_EINVAL
    assert b"at most 1048576 pairs" in L.logbessel_last_error()
    assert L.logbessel_k_noalloc(B.LB_F32, t.data_ptr(), 0, t.data_ptr(), t.data_ptr(), 4, 0, None) == B.LB_ENOTSUP
