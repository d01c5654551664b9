"""logbessel_k_noalloc, the entry point that allocates no device memory
(for callers that cannot let a library allocate: fixed memory budgets,
latency-critical loops, frameworks that own all device memory), against the
allocating logbessel_k on the same inputs, on two calls in a row."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_08729_gb300 import _binding as B
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 4e-15      # the FP64 tolerance of the parity tests
MAX_PAIRS = 1 << 20


def _lib():
    L = B.lib()
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.logbessel_k_noalloc.argtypes = [i32, vp, i64, vp, vp, i64, i32, vp]
    L.logbessel_k_noalloc.restype = i32
    return L


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
        err = np.abs(a - b) / np.maximum(np.abs(b), 1.0)
        assert err.max() <= TOL64, (seed, err.max())


def test_noalloc_rejects_oversized_calls(cuda):
    L = _lib()
    t = torch.ones(4, dtype=torch.float64, device=cuda)
    st = L.logbessel_k_noalloc(B.LB_F64, t.data_ptr(), 0, t.data_ptr(), t.data_ptr(), MAX_PAIRS + 1, 0, None)
    assert st == B.LB_EINVAL
    assert b"at most 1048576 pairs" in L.logbessel_last_error()
    assert L.logbessel_k_noalloc(B.LB_F32, t.data_ptr(), 0, t.data_ptr(), t.data_ptr(), 4, 0, None) == B.LB_ENOTSUP
