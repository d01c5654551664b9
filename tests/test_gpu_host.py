"""End-to-end entry point on host buffers (chunked copy/compute pipeline)
against the device entry points."""
import numpy as np
import pytest
import torch

import paper_2409_08729_gb300 as lb
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _close(a, b, tol):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    same = (a == b) | (np.isnan(a) & np.isnan(b))
    with np.errstate(invalid="ignore"):
        rel = np.abs(a - b) / np.maximum(1.0, np.abs(b))
    return bool(np.all(same | (rel <= tol)))


@pytest.mark.parametrize("fn", ["log_i", "log_k", "log_i_dx", "log_k_dx"])
def test_host_matches_device(cuda, fn):
    v, x = W.robust_pairs(300001, seed=12, vmax=1e4, xmin=1e-5, xmax=1e4)
    got = lb.host_eval(fn, v, x, chunk=65536)             # several chunks, ragged tail
    dev = getattr(lb, fn)(torch.tensor(v, device=cuda), torch.tensor(x, device=cuda)).cpu().numpy()
    assert _close(got, dev, 4e-15 if "dx" not in fn else 2e-14)


@pytest.mark.parametrize("fn", ["log_i", "log_k"])
def test_host_fp32_and_scalar_order(cuda, fn):
    x = np.exp(np.random.default_rng(3).uniform(np.log(1e-3), np.log(1e3), 100000)).astype(np.float32)
    got = lb.host_eval(fn, np.float32(2.5), x, chunk=30000)
    dev = getattr(lb, fn)(2.5, torch.tensor(x, device=cuda)).cpu().numpy()
    assert _close(got, dev, 2e-6)
    xp = torch.from_numpy(x).pin_memory()
    got2 = lb.host_eval(fn, torch.tensor([2.5], dtype=torch.float32), xp)
    assert _close(got2.numpy(), dev, 2e-6)


def test_host_buffers_kept_and_released(cuda):
    """The device buffer and streams outlive a call: a smaller call reuses
    them, a larger chunk grows them, host_release frees them and the next
    call makes them again; chunk edges on tile boundaries give the same bits."""
    v, x = W.robust_pairs(200001, seed=21, vmax=1e3, xmin=1e-4, xmax=1e3)
    a = lb.host_eval("log_k", v, x, chunk=65536)
    b = lb.host_eval("log_k", v[:1000], x[:1000])
    c = lb.host_eval("log_k", v, x, chunk=1 << 20)
    lb.host_release()
    d = lb.host_eval("log_k", v, x, chunk=65536)
    lb.host_release()
    lb.host_release()
    e = lb.host_eval("log_i", 7.0, x, chunk=131072)
    ref_b = lb.log_k(torch.tensor(v[:1000], device=cuda), torch.tensor(x[:1000], device=cuda)).cpu().numpy()
    ref_e = lb.log_i(7.0, torch.tensor(x, device=cuda)).cpu().numpy()
    assert np.array_equal(a, c, equal_nan=True)
    assert np.array_equal(a, d, equal_nan=True)
    assert np.array_equal(b, ref_b, equal_nan=True)
    assert np.array_equal(e, ref_e, equal_nan=True)
