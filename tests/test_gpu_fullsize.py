"""The paper-shaped sweep at its full size, in the launch configuration the
benchmark times: for each order v = 2^0..2^10, 20M arguments x ~ U[1, 100]
in one call with a scalar order, and one mixed-order call over all 220M
pairs.  Checked on sampled outputs against the oracle, and at every element
through properties that hold at any size: finiteness, monotonicity in the
order (log I decreases and log K increases with v at fixed x > 0), and the
agreement of the mixed-order call with the per-order calls wherever the
mixed call drew the same order."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_08729_gb300 as lb
from paper_2409_08729_gb300 import _binding as B
from paper_2409_08729_gb300.workloads import SWEEP_ORDERS, sweep_device

pytestmark = pytest.mark.gpu

N_PER_ORDER = 20_000_000
TOL64 = 4e-15


@pytest.mark.parametrize("kind", ["i", "k"])
def test_full_size_sweep(cuda, kind):
    nv = len(SWEEP_ORDERS)
    n1 = N_PER_ORDER
    x_all, v_mixed = sweep_device(n1, seed=1234, device=cuda)
    orders = torch.tensor(SWEEP_ORDERS, dtype=torch.float64, device=cuda)
    per = torch.empty_like(x_all)
    mix = torch.empty_like(x_all)
    L = B.lib()
    fn = L.logbessel_i if kind == "i" else L.logbessel_k
    sp = torch.cuda.current_stream(cuda).cuda_stream
    for k in range(nv):
        B.check(fn(B.LB_F64, orders[k:k + 1].data_ptr(), 0, x_all[k * n1:(k + 1) * n1].data_ptr(),
                   per[k * n1:(k + 1) * n1].data_ptr(), n1, 0, sp))
    B.check(fn(B.LB_F64, v_mixed.data_ptr(), 1, x_all.data_ptr(), mix.data_ptr(), nv * n1, 0, sp))
    torch.cuda.synchronize()
    assert bool(torch.isfinite(per).all()) and bool(torch.isfinite(mix).all())

    # sampled outputs against the oracle
    rng = np.random.default_rng(77)
    idx = rng.integers(0, nv * n1, 3000)
    it = torch.from_numpy(idx).to(cuda)
    xs = x_all[it].cpu().numpy()
    for got, vv in ((per[it].cpu().numpy(), np.asarray(SWEEP_ORDERS)[idx // n1]), (mix[it].cpu().numpy(),
                                                                                     v_mixed[it].cpu().numpy())):
        ref = oracle.log_i(vv, xs) if kind == "i" else oracle.log_k(vv, xs)
        err = oracle.rel_err(got, ref, oracle.error_scale(kind, vv, xs))
        assert err.max() <= TOL64, (err.max(), vv[err.argmax()], xs[err.argmax()])

    # monotone in the order at every x: evaluate order 2^(k+1) on block k's arguments
    nxt = torch.empty(n1, dtype=torch.float64, device=cuda)
    for k in range(nv - 1):
        B.check(fn(B.LB_F64, orders[k + 1:k + 2].data_ptr(), 0, x_all[k * n1:(k + 1) * n1].data_ptr(),
                   nxt.data_ptr(), n1, 0, sp))
        cur = per[k * n1:(k + 1) * n1]
        if kind == "i":
            assert bool((nxt < cur).all()), k
        else:
            assert bool((nxt > cur).all()), k

    # mixed-order call against the per-order calls where it drew block k's order
    block_order = orders.repeat_interleave(n1)
    same = v_mixed == block_order
    assert int(same.sum()) > nv * n1 // 20
    a, b = mix[same], per[same]
    scale = torch.clamp(b.abs(), min=1.0)
    assert float(((a - b).abs() / scale).max()) <= TOL64


@pytest.mark.parametrize("dx", [False, True])
def test_phased_k_integral_queue(cuda, dx):
    """A K call with more fallback pairs than 256 per warp of the K-integral
    grid evaluates its queue in phases, one quadrature-rule class each; the
    same pairs in calls of 2^20 (tile-aligned, too few fallback pairs for
    phases: taken in order) give the same bits, and the phased call meets
    the gate against the oracle on a sample."""
    from paper_2409_08729_gb300.workloads import robust_device
    n = 1 << 23
    v, x = robust_device(n, 41, cuda, vmax=64.0, xmin=1e-8, xmax=40.0)
    reg = lb.classify("k", v, x)
    assert int((reg == B.REGIONS["fallback"]).sum()) > 152 * 4 * 8 * 256 * 2   # phased
    fn = B.lib().logbessel_k_dx if dx else B.lib().logbessel_k
    sp = torch.cuda.current_stream().cuda_stream
    full = torch.empty(n, dtype=torch.float64, device=cuda)
    B.check(fn(B.LB_F64, v.data_ptr(), 1, x.data_ptr(), full.data_ptr(), n, 0, sp))
    part = torch.empty_like(full)
    c = 1 << 20
    for s in range(0, n, c):
        B.check(fn(B.LB_F64, v[s:s + c].data_ptr(), 1, x[s:s + c].data_ptr(), part[s:s + c].data_ptr(), c, 0, sp))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(full.cpu().numpy(), part.cpu().numpy())
    if not dx:
        idx = np.random.default_rng(2).integers(0, n, 3000)
        vs, xs = v.cpu().numpy()[idx], x.cpu().numpy()[idx]
        e = oracle.rel_err(full.cpu().numpy()[idx], oracle.log_k(vs, xs), oracle.error_scale("k", vs, xs))
        assert e.max() < 4e-15, e.max()
