"""Serving benchmark: Poisson arrivals of mixed requests, continuous batching
(lb_server) against direct library calls.

Request mix (sizes log-uniform on [1, max_n] pairs; 50/50 log I and log K;
70 % FP32-mixed, 30 % FP64; v log-uniform on [1e-6, 1e4]; x log-uniform on
[1e-3, 1e4]).  Inputs come from a pool of pairs; each request reads a window
of it: a pinned host pool for host requests (the server copies in and out),
a device pool for device requests (evaluated in place).

Measured, in this order:
  * batched, host requests: closed-loop capacity (everything submitted at
    once), then the same arrival stream at each offered load (x capacity);
  * batched, device requests: the same;
  * direct, one call per request: the library call of every request, inputs
    on the device, back to back on one stream (CUDA events);
  * direct, large calls: each (kind, dtype) of the mix evaluated in one call
    over the whole device pool; the mix's pairs at those rates give the
    throughput of the kernels on this mix with no request boundaries;
  * one call per request at the offered loads (host buffers: copy in, call,
    copy out, FIFO on one stream), on the first `per_call_requests` requests
    of the stream (that arm cannot keep up: its queue grows without bound).
Latency is completion (result in host memory, or in device memory for device
requests) minus arrival.
"""
import time

import numpy as np
import torch

from paper_2409_08729_gb300 import _binding as B
from paper_2409_08729_gb300.serve import Server


def _mix(n_req, seed, max_n):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(0.0, np.log(max_n), n_req))).astype(np.int64)
    sizes = np.clip(sizes, 1, max_n)
    kinds = np.where(rng.random(n_req) < 0.5, 0, 1)
    f32 = rng.random(n_req) < 0.7
    return sizes, kinds, f32


def _pool(n, seed):
    rng = np.random.default_rng(seed)
    v = np.exp(rng.uniform(np.log(1e-6), np.log(1e4), n))
    x = np.exp(rng.uniform(np.log(1e-3), np.log(1e4), n))
    pv64 = torch.from_numpy(v).pin_memory()
    px64 = torch.from_numpy(x).pin_memory()
    return pv64, px64, pv64.float().pin_memory(), px64.float().pin_memory()


def run(n_req=20000, seed=0, max_n=1_000_000, load=0.8, device="cuda", pool_n=1 << 23, out_slots=512,
        per_call_requests=None):
    """One offered load (a float) or several (a sequence): the capacities are
    measured once, then the arrival stream of each load is replayed."""
    loads = [load] if isinstance(load, (int, float)) else list(load)
    res = _run(n_req, seed, max_n, loads, device, pool_n, out_slots, per_call_requests)
    if isinstance(load, (int, float)):
        for arm in ("batched", "batched_device", "per_request_calls"):
            res[arm] = res.pop(arm + "_by_load")[0]
    return res


def _latency_run(srv, n_req, arr, submit, out_slots):
    tickets = [None] * n_req
    st0 = srv.stats()["kernel_launches"]
    start = time.perf_counter()
    for i in range(n_req):
        dt = arr[i] - (time.perf_counter() - start)
        if dt > 0:
            time.sleep(dt)
        if i >= out_slots:
            srv.wait(tickets[i - out_slots], timeout=300)
        tickets[i] = submit(i)
    for t in tickets[-min(out_slots, n_req):]:
        srv.wait(t, timeout=300)
    lat = np.empty(n_req)
    t_first, t_last = np.inf, 0.0
    for i, t in enumerate(tickets):
        done, ts, ta, td = srv.info(t)
        lat[i] = td - ts
        t_first, t_last = min(t_first, ts), max(t_last, td)
        srv.release(t)
    return lat, t_first, t_last, srv.stats()["kernel_launches"] - st0


def _closed_loop(srv, n_req, submit, out_slots):
    t0 = time.perf_counter()
    tickets = []
    for i in range(n_req):
        if i >= out_slots:
            srv.wait(tickets[i - out_slots], timeout=300)
        tickets.append(submit(i))
    for t in tickets[-min(out_slots, n_req):]:
        srv.wait(t, timeout=300)
    dt = time.perf_counter() - t0
    for t in tickets:
        srv.release(t)
    return dt


def _device_shares(d0, d1, ctas, wall):
    """The persistent kernel's CTA time over a run: the share spent running
    items (per item family too) and claiming or waiting for them."""
    span = ctas * wall * 1e9
    busy = {f: d1["busy_ns"][f] - d0["busy_ns"][f] for f in d1["busy_ns"]}
    items = {f: d1["items"][f] - d0["items"][f] for f in d1["items"]}
    return {"ctas": ctas, "busy_share": sum(busy.values()) / span,
            "claim_wait_share": (d1["claim_ns"] - d0["claim_ns"]) / span,
            "busy_share_by_family": {f: b / span for f, b in busy.items() if items[f]},
            "items_by_family": {f: n for f, n in items.items() if n}}


def _time_cuda(fn, stream):
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _run(n_req, seed, max_n, loads, device, pool_n, out_slots, per_call_requests):
    dev = torch.device(device)
    sizes, kinds, f32 = _mix(n_req, seed, max_n)
    pv64, px64, pv32, px32 = _pool(pool_n, seed + 1)
    dv64, dx64, dv32, dx32 = (t.to(dev) for t in (pv64, px64, pv32, px32))
    rng = np.random.default_rng(seed + 2)
    offs = rng.integers(0, pool_n - max_n, n_req)
    out64 = torch.empty((out_slots, max_n), dtype=torch.float64).pin_memory()
    out32 = torch.empty((out_slots, max_n), dtype=torch.float32).pin_memory()
    # device requests write to regions of their own (nothing is copied back,
    # so the client never waits for a region to be free)
    tot64, tot32 = int(sizes[~f32].sum()), int(sizes[f32].sum())
    dout64 = torch.empty(max(tot64, max_n), dtype=torch.float64, device=dev)
    dout32 = torch.empty(max(tot32, max_n), dtype=torch.float32, device=dev)
    dpos = np.zeros(n_req, dtype=np.int64)
    dpos[~f32] = np.concatenate([[0], np.cumsum(sizes[~f32])[:-1]]) if tot64 else 0
    dpos[f32] = np.concatenate([[0], np.cumsum(sizes[f32])[:-1]]) if tot32 else 0

    def host_args(i):
        o, n = int(offs[i]), int(sizes[i])
        if f32[i]:
            return pv32[o:o + n], px32[o:o + n], out32[i % out_slots, :n]
        return pv64[o:o + n], px64[o:o + n], out64[i % out_slots, :n]

    def dev_args(i):
        o, n, p = int(offs[i]), int(sizes[i]), int(dpos[i])
        if f32[i]:
            return dv32[o:o + n], dx32[o:o + n], dout32[p:p + n]
        return dv64[o:o + n], dx64[o:o + n], dout64[p:p + n]

    # raw pointers of every request, so the submitting loop does not inspect tensors
    def ptrs(bufs, out_pos):
        v64, x64, v32, x32, o64, o32 = (b.data_ptr() for b in bufs)
        es = np.where(f32, 4, 8)
        vb = np.where(f32, v32, v64) + offs * es
        xb = np.where(f32, x32, x64) + offs * es
        ob = np.where(f32, o32, o64) + out_pos * es
        return [(("i", "k")[kinds[i]], B.LB_F32 if f32[i] else B.LB_F64, int(vb[i]), int(xb[i]), int(ob[i]),
                 int(sizes[i])) for i in range(n_req)]

    host_ptrs = ptrs((pv64, px64, pv32, px32, out64, out32), (np.arange(n_req) % out_slots) * max_n)
    dev_ptrs = ptrs((dv64, dx64, dv32, dx32, dout64, dout32), dpos)

    total = int(sizes.sum())
    res = {"requests": n_req, "pairs": total,
           "mix": "sizes log-uniform [1, %d]; I/K 50/50; FP32 70%%; v log-uniform [1e-6, 1e4], "
                  "x log-uniform [1e-3, 1e4]" % max_n}
    torch.cuda.synchronize()
    with Server(arena_bytes=16 << 30, max_slots=1024, ctas_per_sm=4, idle_ms=20.0) as srv:
        def sub_host(i):
            k, dt, v, x, o, n = host_ptrs[i]
            return srv.submit_ptr(k, dt, v, 1, x, o, n)

        def sub_dev(i):
            k, dt, v, x, o, n = dev_ptrs[i]
            return srv.submit_ptr(k, dt, v, 1, x, o, n, device=True)

        for i in range(min(64, n_req)):                  # warm-up
            srv.wait(sub_host(i), timeout=120)
            srv.wait(sub_dev(i), timeout=120)
        cap = {}
        # host requests: output rows are reused, so the client waits for the
        # request that last used a row; device requests: everything submitted
        # at once, then waited for
        ctas = torch.cuda.get_device_properties(dev).multi_processor_count * 4
        for arm, sub, slots_ in (("batched", sub_host, out_slots), ("batched_device", sub_dev, n_req + 1)):
            d0 = srv.device_stats()
            wall = _closed_loop(srv, n_req, sub, slots_)
            d1 = srv.device_stats()
            cap[arm] = total / wall
            res[arm + "_capacity_gevals"] = cap[arm] / 1e9
            res[arm + "_time_shares"] = _device_shares(d0, d1, ctas, wall)
        res["capacity_gevals"] = res["batched_capacity_gevals"]
        arrivals = []
        for load in loads:
            rate = load * cap["batched"] / (total / n_req)            # requests per second
            arrivals.append(np.cumsum(rng.exponential(1.0 / rate, n_req)))
        for arm, sub, slots_ in (("batched", sub_host, out_slots), ("batched_device", sub_dev, n_req + 1)):
            res[arm + "_by_load"] = []
            for load in loads:
                # the same arrival pattern, scaled to this arm's own capacity
                arr = arrivals[loads.index(load)] * cap["batched"] / cap[arm]
                lat, t_first, t_last, relaunches = _latency_run(srv, n_req, arr, sub, slots_)
                res[arm + "_by_load"].append({
                    "offered_load": load, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                    "p99_ms": 1e3 * float(np.percentile(lat, 99)), "gevals": total / (t_last - t_first) / 1e9,
                    # the persistent kernel stays resident while work keeps
                    # arriving; it is relaunched only after idling out
                    "persistent_kernel_relaunches": relaunches})
        res["persistent_kernel_launches_since_start"] = srv.stats()["kernel_launches"]

    L = B.lib()
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream

    # direct: one library call per request, device-resident, back to back
    def direct_calls():
        for i in range(n_req):
            v, x, o = dev_args(i)
            fn = L.logbessel_i if kinds[i] == 0 else L.logbessel_k
            B.check(fn(B.LB_F32 if f32[i] else B.LB_F64, v.data_ptr(), 1, x.data_ptr(), o.data_ptr(), int(sizes[i]),
                       0, sp))

    with torch.cuda.stream(stream):
        direct_calls()                                   # warm-up
        t_calls = _time_cuda(direct_calls, stream)
    res["direct_one_call_per_request_gevals"] = total / t_calls / 1e9

    # direct: large calls over the device pool, one per (kind, dtype)
    rates = {}
    with torch.cuda.stream(stream):
        for kind in (0, 1):
            for is32 in (False, True):
                v, x = (dv32, dx32) if is32 else (dv64, dx64)
                o = (dout32 if is32 else dout64)[:pool_n] if (dout32 if is32 else dout64).numel() >= pool_n else \
                    torch.empty(pool_n, dtype=torch.float32 if is32 else torch.float64, device=dev)
                fn = L.logbessel_i if kind == 0 else L.logbessel_k

                def call():
                    B.check(fn(B.LB_F32 if is32 else B.LB_F64, v.data_ptr(), 1, x.data_ptr(), o.data_ptr(), pool_n,
                               0, sp))
                call()
                rates[(kind, is32)] = pool_n / (_time_cuda(call, stream))
    t_groups = sum(float(sizes[(kinds == k) & (f32 == s)].sum()) / rates[(k, s)] for (k, s) in rates)
    res["direct_large_calls_gevals"] = total / t_groups / 1e9
    res["direct_large_call_rates_gevals"] = {"%s_%s" % ("ik"[k], "f32" if s else "f64"): r / 1e9
                                             for (k, s), r in rates.items()}
    res["batched_device_vs_direct_large_calls"] = res["batched_device_capacity_gevals"] / res["direct_large_calls_gevals"]
    res["batched_device_vs_direct_one_call_per_request"] = (res["batched_device_capacity_gevals"]
                                                            / res["direct_one_call_per_request_gevals"])
    del dout64, dout32

    # one library call per request at the offered loads (host buffers), on the
    # first m requests of each arrival stream
    m = n_req if per_call_requests is None else min(n_req, int(per_call_requests))
    sub_total = int(sizes[:m].sum())
    bv64 = torch.empty(max_n, dtype=torch.float64, device=dev)
    bx64 = torch.empty(max_n, dtype=torch.float64, device=dev)
    bo64 = torch.empty(max_n, dtype=torch.float64, device=dev)
    bv32 = torch.empty(max_n, dtype=torch.float32, device=dev)
    bx32 = torch.empty(max_n, dtype=torch.float32, device=dev)
    bo32 = torch.empty(max_n, dtype=torch.float32, device=dev)
    res["per_request_calls_by_load"] = []
    for load, arr in zip(loads, arrivals):
        lat2 = np.empty(m)
        start = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(m):
                dt = arr[i] - (time.perf_counter() - start)
                if dt > 0:
                    time.sleep(dt)
                hv, hx, ho = host_args(i)
                n = int(sizes[i])
                if f32[i]:
                    dv, dx, do, code = bv32, bx32, bo32, B.LB_F32
                else:
                    dv, dx, do, code = bv64, bx64, bo64, B.LB_F64
                dv[:n].copy_(hv, non_blocking=True)
                dx[:n].copy_(hx, non_blocking=True)
                fn = L.logbessel_i if kinds[i] == 0 else L.logbessel_k
                B.check(fn(code, dv.data_ptr(), 1, dx.data_ptr(), do.data_ptr(), n, 0, sp))
                ho.copy_(do[:n], non_blocking=True)
                stream.synchronize()
                lat2[i] = (time.perf_counter() - start) - arr[i]
        span = (time.perf_counter() - start) - arr[0]
        res["per_request_calls_by_load"].append({
            "offered_load": load, "requests": m, "p50_ms": 1e3 * float(np.percentile(lat2, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat2, 99)), "gevals": sub_total / span / 1e9})
    return res


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Serving benchmark (continuous batching vs direct calls)")
    ap.add_argument("--requests", type=int, default=100_000)
    ap.add_argument("--per-call-requests", type=int, default=10_000)
    ap.add_argument("--loads", default="0.5,0.8,0.95")
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    from paper_2409_08729_gb300 import build_library
    build_library()
    print(json.dumps(run(n_req=a.requests, seed=a.seed, load=[float(t) for t in a.loads.split(",")],
                         per_call_requests=a.per_call_requests)), flush=True)
