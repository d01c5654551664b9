"""FP32-mixed path against the FP64 oracle: err <= 2e-6 of the error scale
(same metric as the FP64 gate, evaluated at the float inputs)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_08729_gb300 as lb
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL32 = 2e-6


def _run32(kind, v, x, dev):
    tv = torch.tensor(v, dtype=torch.float32, device=dev)
    tx = torch.tensor(x, dtype=torch.float32, device=dev)
    out = (lb.log_i if kind == "i" else lb.log_k)(tv, tx)
    reg = lb.classify(kind, tv, tx).cpu().numpy()
    return out.cpu().numpy().astype(np.float64), reg


def _check(kind, v, x, dev):
    v = v.astype(np.float32).astype(np.float64)
    x = x.astype(np.float32).astype(np.float64)
    got, reg = _run32(kind, v, x, dev)
    ref = oracle.log_i(v, x) if kind == "i" else oracle.log_k(v, x)
    ok = np.isfinite(ref)
    scale = np.ones_like(ref)
    scale[ok] = oracle.error_scale(kind, v[ok], x[ok])
    err = oracle.rel_err(got, ref, scale)
    msgs = []
    for name, rid in lb.REGIONS.items():
        sel = reg == rid
        if sel.any():
            msgs.append("%s: n=%d max %.2e" % (name, sel.sum(), err[sel].max()))
    bad = np.flatnonzero(~(err <= TOL32))
    if bad.size:
        i = bad[np.argmax(err[bad])]
        pytest.fail("FP32 log %s: %d/%d above %.0e; worst %.3e at v=%r x=%r (got %r ref %r); %s" % (
            kind.upper(), bad.size, err.size, TOL32, err[i], v[i], x[i], got[i], ref[i], "; ".join(msgs)))
    return err


@pytest.mark.parametrize("kind", ["i", "k"])
def test_sweep(cuda, kind):
    v, x = W.sweep_pairs(5000, seed=0)
    _check(kind, v, x, cuda)


@pytest.mark.parametrize("kind", ["i", "k"])
def test_robust(cuda, kind):
    v, x = W.robust_pairs(30000, seed=31)
    _check(kind, v, x, cuda)


@pytest.mark.parametrize("kind", ["i", "k"])
def test_boundaries(cuda, kind):
    v, x = W.boundary_pairs(seed=9, per_edge=12)
    _check(kind, v, x, cuda)


@pytest.mark.parametrize("kind", ["i", "k"])
def test_ragged(cuda, kind):
    for n in (1, 33, 1025, 5000):
        v, x = W.robust_pairs(n, seed=n + 1, vmax=1e3, xmin=1e-4, xmax=1e3)
        _check(kind, v, x, cuda)


@pytest.mark.parametrize("kind", ["i", "k"])
def test_tiny_arguments(cuda, kind):
    rng = np.random.default_rng(19)
    v = rng.uniform(0, 0.6, 6000)
    x = np.exp(rng.uniform(np.log(1e-37), np.log(1e-2), 6000))
    _check(kind, v, x, cuda)


@pytest.mark.parametrize("kind", ["i", "k"])
def test_wider_expansion_ranges(cuda, kind):
    """Values take mu_20 and U_13 below the shared thresholds in FP32 too:
    dense random pairs over x in (13, 30], v up to 16."""
    rng = np.random.default_rng(23)
    v = rng.uniform(0.0, 16.0, 20000)
    x = rng.uniform(13.0, 30.0, 20000)
    _check(kind, v, x, cuda)
