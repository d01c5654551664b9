"""Serving benchmark: Poisson arrivals of mixed requests, continuous batching
(lb_server) against one library call per request.

Request mix (sizes log-uniform on [1, max_n] pairs; 50/50 log I and log K;
70 % FP32-mixed, 30 % FP64; v log-uniform on [1e-6, 1e4]; x log-uniform on
[1e-3, 1e4]).  Inputs come from a pinned host pool; each request reads a
window of it.  First the closed-loop capacity of the server is measured
(all requests submitted at once), then both systems receive the same
arrival times at an offered load of `load` x capacity.  Latency is
completion (result in host memory) minus arrival.
"""
import threading
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


def run(n_req=20000, seed=0, max_n=1_000_000, load=0.8, device="cuda", pool_n=1 << 23, out_slots=512):
    """One offered load (a float) or several (a sequence): the capacity is
    measured once, then both systems run the arrival stream of each load."""
    loads = [load] if isinstance(load, (int, float)) else list(load)
    res = _run(n_req, seed, max_n, loads, device, pool_n, out_slots)
    if isinstance(load, (int, float)):
        res["batched"] = res.pop("batched_by_load")[0]
        res["per_request_calls"] = res.pop("per_request_calls_by_load")[0]
    return res


def _run(n_req, seed, max_n, loads, device, pool_n, out_slots):
    dev = torch.device(device)
    sizes, kinds, f32 = _mix(n_req, seed, max_n)
    pv64, px64, pv32, px32 = _pool(pool_n, seed + 1)
    rng = np.random.default_rng(seed + 2)
    offs = rng.integers(0, pool_n - max_n, n_req)
    out64 = torch.empty((out_slots, max_n), dtype=torch.float64).pin_memory()
    out32 = torch.empty((out_slots, max_n), dtype=torch.float32).pin_memory()

    def args_of(i):
        o, n = int(offs[i]), int(sizes[i])
        if f32[i]:
            return pv32[o:o + n], px32[o:o + n], out32[i % out_slots, :n]
        return pv64[o:o + n], px64[o:o + n], out64[i % out_slots, :n]

    total = int(sizes.sum())
    res = {"requests": n_req, "pairs": total, "mix": "sizes log-uniform [1, %d]; I/K 50/50; FP32 70%%" % max_n}
    with Server(arena_bytes=8 << 30, max_slots=256, ctas_per_sm=4, idle_ms=20.0) as srv:
        # warm-up
        for i in range(min(64, n_req)):
            srv.wait(srv.submit("ik"[kinds[i]], *args_of(i)), timeout=120)
        # closed-loop capacity: everything submitted at once (in-flight slots bound the reuse of out rows)
        t0 = time.perf_counter()
        tickets = []
        for i in range(n_req):
            if i >= out_slots:
                srv.wait(tickets[i - out_slots], timeout=300)
            tickets.append(srv.submit("ik"[kinds[i]], *args_of(i)))
        for t in tickets[-out_slots:]:
            srv.wait(t, timeout=300)
        cap = total / (time.perf_counter() - t0)
        for t in tickets:
            srv.release(t)
        res["capacity_gevals"] = cap / 1e9
        res["batched_by_load"] = []
        arrivals = []
        for load in loads:
            # open loop, Poisson arrivals at load x capacity (in pairs per second)
            rate = load * cap / (total / n_req)                # requests per second
            arr = np.cumsum(rng.exponential(1.0 / rate, n_req))
            arrivals.append(arr)
            tickets = [None] * n_req
            st0 = srv.stats()["kernel_launches"]
            start = time.perf_counter()
            for i in range(n_req):
                dt = arr[i] - (time.perf_counter() - start)
                if dt > 0:
                    time.sleep(dt)
                if i >= out_slots:
                    srv.wait(tickets[i - out_slots], timeout=300)
                tickets[i] = srv.submit("ik"[kinds[i]], *args_of(i))
            for t in tickets[-out_slots:]:
                srv.wait(t, timeout=300)
            lat = np.empty(n_req)
            t_first, t_last = np.inf, 0.0
            for i, t in enumerate(tickets):
                done, ts, ta, td = srv.info(t)
                lat[i] = td - ts
                t_first, t_last = min(t_first, ts), max(t_last, td)
                srv.release(t)
            res["batched_by_load"].append({
                "offered_load": load, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "gevals": total / (t_last - t_first) / 1e9,
                # the persistent kernel started before this run stays resident
                # while work keeps arriving; it is relaunched only after idling out
                "persistent_kernel_relaunches": srv.stats()["kernel_launches"] - st0,
                "persistent_kernel_launches_since_start": srv.stats()["kernel_launches"]})

    # one library call per request, same arrivals, one stream, FIFO
    L = B.lib()
    stream = torch.cuda.Stream(dev)
    dv64 = torch.empty(max_n, dtype=torch.float64, device=dev)
    dx64 = torch.empty(max_n, dtype=torch.float64, device=dev)
    do64 = torch.empty(max_n, dtype=torch.float64, device=dev)
    dv32 = torch.empty(max_n, dtype=torch.float32, device=dev)
    dx32 = torch.empty(max_n, dtype=torch.float32, device=dev)
    do32 = torch.empty(max_n, dtype=torch.float32, device=dev)
    res["per_request_calls_by_load"] = []
    for load, arr in zip(loads, arrivals):
        lat2 = np.empty(n_req)
        start = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(n_req):
                dt = arr[i] - (time.perf_counter() - start)
                if dt > 0:
                    time.sleep(dt)
                hv, hx, ho = args_of(i)
                n = int(sizes[i])
                if f32[i]:
                    dv, dx, do, code = dv32, dx32, do32, B.LB_F32
                else:
                    dv, dx, do, code = dv64, dx64, do64, B.LB_F64
                dv[:n].copy_(hv, non_blocking=True)
                dx[:n].copy_(hx, non_blocking=True)
                fn = L.logbessel_i if kinds[i] == 0 else L.logbessel_k
                B.check(fn(code, dv.data_ptr(), 1, dx.data_ptr(), do.data_ptr(), n, 0, stream.cuda_stream))
                ho.copy_(do[:n], non_blocking=True)
                stream.synchronize()
                lat2[i] = (time.perf_counter() - start) - arr[i]
        span = (time.perf_counter() - start) - arr[0]
        res["per_request_calls_by_load"].append({
            "offered_load": load, "p50_ms": 1e3 * float(np.percentile(lat2, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat2, 99)), "gevals": total / span / 1e9})
    return res


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Serving benchmark (continuous batching vs one call per request)")
    ap.add_argument("--requests", type=int, default=100_000)
    ap.add_argument("--loads", default="0.5,0.8,0.95")
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    from paper_2409_08729_gb300 import build_library
    build_library()
    print(json.dumps(run(n_req=a.requests, seed=a.seed, load=[float(t) for t in a.loads.split(",")])), flush=True)
