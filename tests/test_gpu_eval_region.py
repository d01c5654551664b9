"""One expression forced for every pair (logbessel_eval_region): inside the
region the dispatch assigns, it gives the dispatched result bit for bit;
outside, the K integral stays finite and accurate far beyond its region
(its sums are shifted by the exact maximum, whatever the size of the
exponents)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_08729_gb300 as lb
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["i", "k"])
def test_forced_equals_dispatch_inside(cuda, kind):
    """U_K and the K integral are per pair: bit for bit.  mu_20 and the
    series sum the warp's largest term count, so the two agree to rounding
    (within the 4e-15 gate, in the error metric's units)."""
    v, x = W.robust_pairs(200000, seed=31, vmax=2e3, xmin=1e-4, xmax=2e3)
    vt, xt = torch.tensor(v, device=cuda), torch.tensor(x, device=cuda)
    reg = lb.classify(kind, vt, xt).cpu().numpy()
    full = (lb.log_i if kind == "i" else lb.log_k)(vt, xt).cpu().numpy()
    checked = 0
    for name in ("mu20", "u13", "fallback", "u4", "u6", "u9"):
        sel = reg == lb.REGIONS[name]
        if not sel.any():
            continue
        idx = torch.tensor(np.flatnonzero(sel), device=cuda)
        got = lb.eval_region(kind, name, vt[idx], xt[idx]).cpu().numpy()
        if name.startswith("u") or (kind == "k" and name == "fallback"):
            np.testing.assert_array_equal(got, full[sel])
        else:
            # two valid evaluations, each within the gate of the oracle: the
            # error metric's units (scale max(|f|, c), c = max(1, |x df/dx|, |v df/dv|))
            e = oracle.rel_err(got, full[sel], oracle.error_scale(kind, v[sel], x[sel]))
            assert e.max() < 4e-15, (name, e.max())
        checked += int(sel.sum())
    assert checked > 100000


def test_k_integral_far_outside(cuda):
    """The K integral's Gauss rules forced far outside their region, where
    the node exponents reach 1e9: finite everywhere (the sums are shifted by
    the exact maximum), and within 1e-14 of the oracle wherever the rule
    still resolves the integrand (a 30-digit sum of the same tables gives
    1e-17 there; v = 100, x = 150 is beyond the Laguerre rule: 9e-3)."""
    v = np.array([0.3, 1.0, 3.0, 12.0, 40.0, 100.0, 16.0, 16.0])
    x = np.array([1e3, 1e4, 2e3, 5e2, 60.0, 150.0, 1e5, 1e8])
    got = lb.eval_region("k", "fallback", torch.tensor(v, device=cuda), torch.tensor(x, device=cuda)).cpu().numpy()
    assert np.all(np.isfinite(got))
    err = oracle.rel_err(got, oracle.log_k(v, x), oracle.error_scale("k", v, x))
    resolved = np.arange(v.size) != 5
    assert err[resolved].max() < 1e-14, err
