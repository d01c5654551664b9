"""Caller-workspace K entry points: same results as logbessel_k /
logbessel_k_dx, in several passes when the workspace holds fewer pairs than
the call."""
import numpy as np
import pytest
import torch

from paper_2409_08729_gb300 import _binding as B
from paper_2409_08729_gb300.workloads import robust_pairs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("ws_pairs", [2048, 5000, 1 << 20])
def test_k_ws_matches_logbessel_k(cuda, dtype, ws_pairs):
    v, x = robust_pairs(300_000, seed=41)
    vt = torch.tensor(v, dtype=dtype, device=cuda)
    xt = torch.tensor(x, dtype=dtype, device=cuda)
    n = vt.numel()
    code = B.LB_F64 if dtype == torch.float64 else B.LB_F32
    L = B.lib()
    sp = torch.cuda.current_stream(cuda).cuda_stream
    ref = torch.empty_like(xt)
    B.check(L.logbessel_k(code, vt.data_ptr(), 1, xt.data_ptr(), ref.data_ptr(), n, 0, sp))
    nbytes = 256 + 4 * ws_pairs
    ws = torch.empty(nbytes, dtype=torch.uint8, device=cuda)
    assert ws.data_ptr() % 256 == 0
    got = torch.empty_like(xt)
    B.check(L.logbessel_k_ws(code, vt.data_ptr(), 1, xt.data_ptr(), got.data_ptr(), n, 0, ws.data_ptr(), nbytes, sp))
    torch.testing.assert_close(got, ref, rtol=0, atol=0, equal_nan=True)
    if dtype == torch.float64:
        ref_dx = torch.empty_like(xt)
        B.check(L.logbessel_k_dx(code, vt.data_ptr(), 1, xt.data_ptr(), ref_dx.data_ptr(), n, 0, sp))
        got_dx = torch.empty_like(xt)
        B.check(L.logbessel_k_dx_ws(code, vt.data_ptr(), 1, xt.data_ptr(), got_dx.data_ptr(), n, 0, ws.data_ptr(),
                                    nbytes, sp))
        torch.testing.assert_close(got_dx, ref_dx, rtol=0, atol=0, equal_nan=True)
