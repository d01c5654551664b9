"""Adjoint kernels d/dx log I_v(x), d/dx log K_v(x) against the oracle's
Bessel-ratio derivative (DLMF 10.29.2) and against central finite differences
of the forward kernels; autograd through the torch Function."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_08729_gb300 as lb
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu
# Relative tolerance of the FP64 derivative, the gate of the values (the paper
# gives no bound for derivatives).  The derivative rules of the K integral are
# within 1.2e-16 of the oracle's Bessel ratio (error map in test_kquad.py);
# the worst measured end to end on these sets is 2.1e-15.
TOL_DX = 4e-15


def _dx(kind, v, x, dev, scalar_v=False):
    tx = torch.tensor(x, dtype=torch.float64, device=dev)
    tv = float(v[0]) if scalar_v else torch.tensor(v, dtype=torch.float64, device=dev)
    fn = lb.log_i_dx if kind == "i" else lb.log_k_dx
    out = fn(tv, tx)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check(kind, v, x, got, tol=TOL_DX):
    ref = oracle.dlog_i_dx(v, x) if kind == "i" else oracle.dlog_k_dx(v, x)
    # scale: |ref|, floored by the (v+1)/x size of the individual terms
    scale = np.maximum(np.abs(ref), 1e-300)
    err = np.abs(got - ref) / scale
    bad = np.flatnonzero(~(err <= tol))
    if bad.size:
        i = bad[np.argmax(err[bad])]
        pytest.fail("d/dx log %s: %d/%d above %.1e; worst %.3e at v=%r x=%r (got %r ref %r)" % (
            kind.upper(), bad.size, err.size, tol, err[i], v[i], x[i], got[i], ref[i]))
    return err


@pytest.mark.parametrize("kind", ["i", "k"])
def test_sweep(cuda, kind):
    v, x = W.sweep_pairs(2000, seed=3)
    _check(kind, v, x, _dx(kind, v, x, cuda))


@pytest.mark.parametrize("kind", ["i", "k"])
def test_robust(cuda, kind):
    v, x = W.robust_pairs(8000, seed=21, vmax=1e4, xmin=1e-5, xmax=1e5)
    _check(kind, v, x, _dx(kind, v, x, cuda))


@pytest.mark.parametrize("kind", ["i", "k"])
def test_boundaries(cuda, kind):
    v, x = W.boundary_pairs(seed=6, per_edge=8)
    _check(kind, v, x, _dx(kind, v, x, cuda))


@pytest.mark.parametrize("kind", ["i", "k"])
def test_finite_differences(cuda, kind):
    """Central differences of the forward kernel: (f(x+h) - f(x-h)) / 2h,
    h = 1e-5 x, truncation ~ h^2 f''' and rounding ~ eps |f| / h."""
    rng = np.random.default_rng(4)
    v = np.exp(rng.uniform(np.log(0.05), np.log(2000.0), 4000))
    x = np.exp(rng.uniform(np.log(0.05), np.log(5000.0), 4000))
    h = 1e-5 * x
    fn = lb.log_i if kind == "i" else lb.log_k
    tv = torch.tensor(v, device=cuda)
    fp = fn(tv, torch.tensor(x + h, device=cuda)).cpu().numpy()
    fm = fn(tv, torch.tensor(x - h, device=cuda)).cpu().numpy()
    fd = (fp - fm) / ((x + h) - (x - h))
    d = _dx(kind, v, x, cuda)
    f0 = fn(tv, torch.tensor(x, device=cuda)).cpu().numpy()
    bound = 1e-8 * np.abs(d) + 4e-16 * np.maximum(1, np.abs(f0)) / h
    assert np.all(np.abs(fd - d) <= bound)


@pytest.mark.parametrize("kind", ["i", "k"])
def test_autograd(cuda, kind):
    v, x = W.sweep_pairs(300, seed=8)
    tx = torch.tensor(x, device=cuda, requires_grad=True)
    tv = torch.tensor(v, device=cuda)
    y = (lb.log_i if kind == "i" else lb.log_k)(tv, tx)
    (y * 2.0).sum().backward()
    ref = 2.0 * _dx(kind, v, x, cuda)
    assert np.array_equal(tx.grad.cpu().numpy(), ref)


def test_domain_edges(cuda):
    v = np.array([0.0, 2.0, 1.0, np.nan, 1.0])
    x = np.array([0.0, 0.0, np.inf, 1.0, -1.0])
    di = _dx("i", v, x, cuda)
    dk = _dx("k", v, x, cuda)
    assert di[0] == 0.0 and di[1] == np.inf and di[2] == 1.0 and np.isnan(di[3]) and np.isnan(di[4])
    assert dk[0] == -np.inf and dk[1] == -np.inf and dk[2] == -1.0 and np.isnan(dk[3]) and np.isnan(dk[4])


def test_k_derivative_tiny_arguments(cuda):
    rng = np.random.default_rng(18)
    v = rng.uniform(0, 0.4, 1500)
    x = np.exp(rng.uniform(np.log(1e-300), np.log(1e-3), 1500))
    _check("k", v, x, _dx("k", v, x, cuda))
