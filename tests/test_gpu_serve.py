"""Serving loop: every served request matches the oracle (FP64 gate 4e-15,
FP32-mixed 2e-6 at its float inputs) and the one-call path, alone and in the
mix; host and device-resident requests; admission by memory; bounded waits;
relaunch after idle."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2409_08729_gb300 as lb
from paper_2409_08729_gb300.serve import Server
from paper_2409_08729_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {np.dtype(np.float64): 4e-15, np.dtype(np.float32): 2e-6}


def _oracle_ok(kind, v, x, o, per_request=256, seed=0):
    """A sample of the request's outputs (all of them for small requests)
    against the oracle at the request's own inputs (float inputs widened
    exactly), in the error metric of the parity tests."""
    n = x.size
    idx = np.arange(n) if n <= per_request else np.random.default_rng(seed).choice(n, per_request, replace=False)
    vv = (v if v.size > 1 else np.broadcast_to(v, x.shape))[idx].astype(np.float64)
    xx = x[idx].astype(np.float64)
    ref = oracle.log_i(vv, xx) if kind == "i" else oracle.log_k(vv, xx)
    err = oracle.rel_err(o[idx].astype(np.float64), ref, oracle.error_scale(kind, vv, xx))
    return float(err.max()) <= TOL[o.dtype], float(err.max())


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
        for i, (k, v, x, o) in enumerate(reqs):
            ok, worst = _oracle_ok(k, v, x, o, seed=i)
            assert ok, (i, k, o.dtype, x.size, worst)
            assert _close(o, _alone(k, v, x, cuda), o.dtype)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["in_flight"] == 0


def _device_requests(reqs, dev):
    out = []
    for k, v, x, o in reqs:
        tv = torch.from_numpy(np.ascontiguousarray(v)).to(dev)
        tx = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        out.append((k, tv, tx, torch.full_like(tx, float("nan"))))
    return out


def test_device_requests_match_oracle(cuda):
    """Requests on device buffers (evaluated in place, nothing copied): every
    result against the oracle on a sample and against the one-call path."""
    reqs = _requests(48, seed=6)
    dreqs = _device_requests(reqs, cuda)
    with Server(arena_bytes=256 << 20, max_slots=32) as srv:
        tickets = [srv.submit_device(k, tv, tx, to) for k, tv, tx, to in dreqs]
        for t in tickets:
            srv.wait(t, timeout=120)
    for i, ((k, v, x, _), (_, tv, tx, to)) in enumerate(zip(reqs, dreqs)):
        o = to.cpu().numpy()
        ok, worst = _oracle_ok(k, v, x, o, seed=100 + i)
        assert ok, (i, k, o.dtype, x.size, worst)
        assert _close(o, _alone(k, v, x, cuda), o.dtype)


def test_host_and_device_requests_together(cuda):
    """Host and device requests submitted interleaved share the device; a
    K-heavy device request (every pair in the integral, all six rule classes)
    is served in the mix and equals the same request served alone."""
    reqs = _requests(30, seed=7)
    rng = np.random.default_rng(7)
    vk = np.concatenate([rng.uniform(0.0, 16.0, 20000), [0.1, 0.3, 1.0, 3.0, 10.0]])
    xk = np.concatenate([np.exp(rng.uniform(np.log(1e-8), np.log(25.0), 20000)), [1e-5, 1e-300, 0.5, 2.0, 24.0]])
    tv, tx = torch.tensor(vk, device=cuda), torch.tensor(xk, device=cuda)
    heavy_mix, heavy_alone = torch.empty_like(tx), torch.empty_like(tx)
    with Server(arena_bytes=128 << 20, max_slots=16) as srv:
        srv.wait(srv.submit_device("k", tv, tx, heavy_alone), timeout=120)
        ts = []
        for i, (k, v, x, o) in enumerate(reqs):
            ts.append(srv.submit(k, v, x, o))
            if i == 10:
                ts.append(srv.submit_device("k", tv, tx, heavy_mix))
        for t in ts:
            srv.wait(t, timeout=120)
    assert torch.equal(heavy_mix, heavy_alone)
    ok, worst = _oracle_ok("k", vk, xk, heavy_mix.cpu().numpy(), per_request=2000)
    assert ok, worst
    for i, (k, v, x, o) in enumerate(reqs):
        ok, worst = _oracle_ok(k, v, x, o, seed=200 + i)
        assert ok, (i, worst)


def test_device_request_waits_for_its_inputs(cuda):
    """A device request starts only once its ready event has completed: the
    inputs written on a side stream after a long kernel are the ones used."""
    n = 300000
    v, x = W.robust_pairs(n, seed=8, vmax=1e4, xmin=1e-3, xmax=1e4)
    tv = torch.zeros(n, dtype=torch.float64, device=cuda)
    tx = torch.ones(n, dtype=torch.float64, device=cuda)
    out = torch.empty_like(tx)
    side = torch.cuda.Stream(cuda)
    side.wait_stream(torch.cuda.current_stream(cuda))     # after the fills above
    hv, hx = torch.from_numpy(v).pin_memory(), torch.from_numpy(x).pin_memory()
    with Server(arena_bytes=64 << 20, max_slots=4) as srv:
        with torch.cuda.stream(side):
            torch.cuda._sleep(50_000_000)          # keep the side stream busy for a while
            tv.copy_(hv, non_blocking=True)
            tx.copy_(hx, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(side)
        t = srv.submit_device("i", tv, tx, out, ready=ready)
        srv.wait(t, timeout=120)
    ok, worst = _oracle_ok("i", v, x, out.cpu().numpy(), per_request=2000)
    assert ok, worst


def test_one_at_a_time_equals_mix(cuda):
    """Each request served alone and served in the mix gives the same bits
    (a pair's result does not depend on the tile or window it shares)."""
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
        assert np.array_equal(o, a, equal_nan=True)


def test_admission_by_memory(cuda):
    """Total request memory far above the arena: requests wait for memory,
    all complete, and results are right."""
    reqs = _requests(40, seed=3, max_n=100000)
    with Server(arena_bytes=4 << 20, max_slots=64) as srv:
        ts = [srv.submit(k, v, x, o) for k, v, x, o in reqs]
        for t in ts:
            srv.wait(t, timeout=120)
        for i, (k, v, x, o) in enumerate(reqs):
            assert _close(o, _alone(k, v, x, cuda), o.dtype)
            ok, worst = _oracle_ok(k, v, x, o, per_request=64, seed=300 + i)
            assert ok, (i, worst)


def test_rejections_and_timeout(cuda):
    with Server(arena_bytes=1 << 20, max_slots=4) as srv:
        big = np.ones(200000)
        with pytest.raises(lb.LogBesselError) as e:
            srv.submit("i", big, big, np.empty_like(big))
        assert "arena" in str(e.value)
        with pytest.raises(lb.LogBesselError):
            srv.submit("q", big[:4], big[:4], np.empty(4))
        # K integral heavy; 15000 pairs: 360 KB of v, x, out and 360 KB of class queues
        v, x = W.robust_pairs(15000, seed=4, vmax=16, xmin=1e-3, xmax=25)
        o = np.empty_like(x)
        t = srv.submit("k", v, x, o)
        try:
            srv.wait(t, timeout=1e-6)
        except lb.LogBesselError as err:
            assert err.status == 4      # LB_ETIMEOUT; the request stays queued
        srv.wait(t, timeout=60)
        assert _close(o, _alone("k", v, x, cuda), np.float64)
        # a device request whose K queues alone exceed the arena is rejected too
        tb = torch.ones(50000, dtype=torch.float64, device=cuda)
        with pytest.raises(lb.LogBesselError) as e:
            srv.submit_device("k", tb, tb, torch.empty_like(tb))
        assert "arena" in str(e.value)


def test_relaunch_after_idle(cuda):
    with Server(arena_bytes=16 << 20, max_slots=4, idle_ms=5.0) as srv:
        v, x = W.robust_pairs(5000, seed=5)
        o1, o2 = np.empty_like(x), np.empty_like(x)
        srv.wait(srv.submit("i", v, x, o1), timeout=30)
        time.sleep(0.1)                  # every thread block has exited by now
        srv.wait(srv.submit("i", v, x, o2), timeout=30)
        assert srv.stats()["kernel_launches"] >= 2
        assert np.array_equal(o1, o2)


def test_device_time_accounts(cuda):
    """The persistent kernel's device time accounts: the items of each family
    are counted (tiles per item as the scheduler splits them), their busy time
    is positive, and the counters only grow."""
    rng = np.random.default_rng(11)
    x_i = torch.tensor(rng.uniform(1.0, 100.0, 5000), device=cuda)             # 5 tiles: 5 FP64 items
    # 8 tiles, 2 items; x > 30 at v = 5: mu_20 only, no integral
    x_k32 = torch.tensor(rng.uniform(31.0, 100.0, 8000), device=cuda, dtype=torch.float32)
    v_kf = torch.tensor(rng.uniform(0.0, 16.0, 4000), device=cuda)             # every pair in the integral
    x_kf = torch.tensor(rng.uniform(0.5, 25.0, 4000), device=cuda)
    with Server(arena_bytes=64 << 20, max_slots=8) as srv:
        d0 = srv.device_stats()
        assert d0["claim_ns"] == 0 and sum(d0["items"].values()) == 0
        ts = [srv.submit_device("i", torch.tensor([3.0], device=cuda, dtype=torch.float64), x_i,
                                torch.empty_like(x_i)),
              srv.submit_device("k", torch.tensor([5.0], device=cuda, dtype=torch.float32), x_k32,
                                torch.empty_like(x_k32)),
              srv.submit_device("k", v_kf, x_kf, torch.empty_like(x_kf))]
        for t in ts:
            srv.wait(t, timeout=120)
        time.sleep(0.05)                           # the last item's time is booked at the next claim
        d1 = srv.device_stats()
    items, busy = d1["items"], d1["busy_ns"]
    assert items["tiles_i_f64"] == 5 and busy["tiles_i_f64"] > 0
    assert items["tiles_k_f32"] == 2 and busy["tiles_k_f32"] > 0
    assert items["tiles_k_f64"] == 4 and busy["tiles_k_f64"] > 0
    kint = [f for f in items if f.startswith("kint_f64")]
    assert sum(items[f] for f in kint) >= 1 and sum(busy[f] for f in kint) > 0
    assert items["tiles_i_f32"] == 0 and items["kint_f32"] == 0
    assert d1["claim_ns"] > d0["claim_ns"]
