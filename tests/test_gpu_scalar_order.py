"""Calls with one order for all arguments (v_stride 0) take per-block
constants (the mu_20 coefficients, series ratios, U_K polynomials in t, the
K integral's node positions).  They must agree with the same call given the
order as a vector, and with the oracle, in every region and at the edges."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_08729_gb300 import _binding as B

pytestmark = pytest.mark.gpu

ORDERS = [0.0, 1e-300, 1e-6, 0.3, 0.5, 0.7000001, 1.0, 2.5, 5.0, 12.6964, 13.6, 16.0, 16.0000001, 20.0, 28.5, 70.5,
          230.5, 1e3, 1e5]


def _call(fn, code, v, stride, x, dev):
    out = torch.empty_like(x)
    sp = torch.cuda.current_stream(dev).cuda_stream
    B.check(fn(code, v.data_ptr(), stride, x.data_ptr(), out.data_ptr(), x.numel(), 0, sp))
    return out


@pytest.mark.parametrize("kind", ["i", "k"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_scalar_order_matches_vector_order(cuda, kind, dtype):
    rng = np.random.default_rng(51)
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-6), np.log(1e5), 6000)), rng.uniform(0.1, 100, 3000),
                        [0.0, 1e-300, 25.0, 30.0, 59.6925, 1e5]])
    xt = torch.tensor(x, dtype=dtype, device=cuda)
    L = B.lib()
    fn = L.logbessel_i if kind == "i" else L.logbessel_k
    code = B.LB_F64 if dtype == torch.float64 else B.LB_F32
    tol = 4e-15 if dtype == torch.float64 else 2e-6
    for v in ORDERS:
        vs = torch.tensor([v], dtype=dtype, device=cuda)
        vv = torch.full_like(xt, v)
        a = _call(fn, code, vs, 0, xt, cuda).double().cpu().numpy()
        b = _call(fn, code, vv, 1, xt, cuda).double().cpu().numpy()
        same_inf = np.isinf(a) & (a == b)
        both_nan = np.isnan(a) & np.isnan(b)
        fin = ~(same_inf | both_nan)
        assert np.all(np.isfinite(a[fin])) and np.all(np.isfinite(b[fin])), v
        scale = np.maximum(np.abs(b[fin]), 1.0)
        assert np.max(np.abs(a[fin] - b[fin]) / scale) <= tol, (v, kind)
        if dtype == torch.float64:
            vf = np.full(x.shape, v)
            ref = oracle.log_i(vf, x) if kind == "i" else oracle.log_k(vf, x)
            ok = np.isfinite(ref) & (x > 0) & (x < 1e8)
            err = oracle.rel_err(a[ok], ref[ok], oracle.error_scale(kind, vf[ok], x[ok]))
            assert err.max() <= tol, (v, kind, err.max(), x[ok][err.argmax()])
