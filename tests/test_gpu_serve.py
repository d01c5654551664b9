"""Serving loop: results equal the one-call path alone and in the mix;
admission by memory; bounded waits; relaunch after idle."""
import time

import numpy as np
import pytest
import torch

import paper_2409_08729_gb300 as lb
from paper_2409_08729_gb300.serve import Server
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _requests(n_req, seed, max_n=60000):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_req):
        n = int(np.exp(rng.uniform(0, np.log(max_n))))
        kind = "i" if rng.random() < 0.5 else "k"
        dt = np.float32 if rng.random() < 0.7 else np.float64
        v, x = W.robust_pairs(n, seed=seed * 1000 + i, vmax=1e4, xmin=1e-3, xmax=1e4)
        if rng.random() < 0.2:
            v = v[:1]                      # one order for the whole request
        reqs.append((kind, v.astype(dt), x.astype(dt), np.empty(n, dtype=dt)))
    return reqs


def _alone(kind, v, x, dev):
    tv = torch.tensor(v, device=dev) if v.size > 1 else float(v[0])
    tx = torch.tensor(x, device=dev)
    return (lb.log_i if kind == "i" else lb.log_k)(tv, tx).cpu().numpy()


def _close(a, b, dt):
    tol = 4e-15 if dt == np.float64 else 2e-6
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    same = (a64 == b64) | (np.isnan(a64) & np.isnan(b64))
    with np.errstate(invalid="ignore"):
        rel = np.abs(a64 - b64) / np.maximum(1.0, np.abs(b64))
    return bool(np.all(same | (rel <= tol)))


def test_mix_equals_alone(cuda):
    reqs = _requests(60, seed=1)
    with Server(arena_bytes=256 << 20, max_slots=32) as srv:
        tickets = [srv.submit(k, v, x, o) for k, v, x, o in reqs]
        for t in tickets:
            srv.wait(t, timeout=120)
        for (k, v, x, o) in reqs:
            assert _close(o, _alone(k, v, x, cuda), o.dtype)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["in_flight"] == 0


def test_one_at_a_time_equals_mix(cuda):
    reqs = _requests(12, seed=2, max_n=20000)
    outs_alone = []
    with Server(arena_bytes=64 << 20, max_slots=8) as srv:
        for k, v, x, o in reqs:
            srv.wait(srv.submit(k, v, x, o), timeout=60)
            outs_alone.append(o.copy())
        for k, v, x, o in reqs:
            o[:] = 0
        ts = [srv.submit(k, v, x, o) for k, v, x, o in reqs]
        for t in ts:
            srv.wait(t, timeout=60)
    for (k, v, x, o), a in zip(reqs, outs_alone):
        assert _close(o, a, o.dtype)


def test_admission_by_memory(cuda):
    """Total request memory far above the arena: requests wait for memory,
    all complete, and results are right."""
    reqs = _requests(40, seed=3, max_n=100000)
    with Server(arena_bytes=4 << 20, max_slots=64) as srv:
        ts = [srv.submit(k, v, x, o) for k, v, x, o in reqs]
        for t in ts:
            srv.wait(t, timeout=120)
        for (k, v, x, o) in reqs:
            assert _close(o, _alone(k, v, x, cuda), o.dtype)


def test_rejections_and_timeout(cuda):
    with Server(arena_bytes=1 << 20, max_slots=4) as srv:
        big = np.ones(200000)
        with pytest.raises(lb.LogBesselError) as e:
            srv.submit("i", big, big, np.empty_like(big))
        assert "arena" in str(e.value)
        with pytest.raises(lb.LogBesselError):
            srv.submit("q", big[:4], big[:4], np.empty(4))
        v, x = W.robust_pairs(30000, seed=4, vmax=16, xmin=1e-3, xmax=25)     # K integral heavy
        o = np.empty_like(x)
        t = srv.submit("k", v, x, o)
        try:
            srv.wait(t, timeout=1e-6)
        except lb.LogBesselError as err:
            assert err.status == 4      # LB_ETIMEOUT; the request stays queued
        srv.wait(t, timeout=60)
        assert _close(o, _alone("k", v, x, cuda), np.float64)


def test_relaunch_after_idle(cuda):
    with Server(arena_bytes=16 << 20, max_slots=4, idle_ms=5.0) as srv:
        v, x = W.robust_pairs(5000, seed=5)
        o1, o2 = np.empty_like(x), np.empty_like(x)
        srv.wait(srv.submit("i", v, x, o1), timeout=30)
        time.sleep(0.1)                  # every thread block has exited by now
        srv.wait(srv.submit("i", v, x, o2), timeout=30)
        assert srv.stats()["kernel_launches"] >= 2
        assert np.array_equal(o1, o2)
