"""Robustness/precision sweep: throughput and per-region error of the FP64
and FP32-mixed forms on pairs that span the whole domain.

Workload: n pairs (default 64M), v log-uniform on [1e-6, 1e5] with 1 %
exactly 0 and 1 % exactly 1/2, x log-uniform on [1e-6, 1e5] (v >> x and
x >> v both present); log I and log K over all of them, one call each,
inputs resident on the device (64M pairs = 1 GB of inputs per dtype, far
above L2).  Error: for every region of the tight dispatch, up to `per_region`
outputs drawn at random among that region's pairs are checked against the
oracle (metric |got - ref| / max(|ref|, c), c = max(1, |x df/dx|, |v df/dv|));
the FP32-mixed form is compared with the oracle at its own (rounded) inputs.
"""
import numpy as np
import torch

from paper_2409_08729_gb300 import _binding as B
from paper_2409_08729_gb300 import classify
from paper_2409_08729_gb300.workloads import robust_device

REGION_NAMES = {0: "mu20", 1: "u13", 2: "fallback", 3: "special", 4: "mu3", 5: "u4", 6: "u6", 7: "u9"}


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run(n=64 << 20, seed=3, device="cuda", reps=3, per_region=1000, check=True):
    dev = torch.device(device)
    v, x = robust_device(n, seed, dev)
    v32, x32 = v.float(), x.float()
    L = B.lib()
    sp = torch.cuda.current_stream(dev).cuda_stream
    out = torch.empty((2, n), dtype=torch.float64, device=dev)
    out32 = torch.empty((2, n), dtype=torch.float32, device=dev)

    def f64():
        B.check(L.logbessel_i(B.LB_F64, v.data_ptr(), 1, x.data_ptr(), out[0].data_ptr(), n, 0, sp))
        B.check(L.logbessel_k(B.LB_F64, v.data_ptr(), 1, x.data_ptr(), out[1].data_ptr(), n, 0, sp))

    def f32():
        B.check(L.logbessel_i(B.LB_F32, v32.data_ptr(), 1, x32.data_ptr(), out32[0].data_ptr(), n, 0, sp))
        B.check(L.logbessel_k(B.LB_F32, v32.data_ptr(), 1, x32.data_ptr(), out32[1].data_ptr(), n, 0, sp))

    ms64 = _time(f64, reps)
    ms32 = _time(f32, reps)
    res = {"pairs": n, "workload": "v log-uniform [1e-6, 1e5] (1% 0, 1% 1/2), x log-uniform [1e-6, 1e5]; "
                                   "log I + log K, one call each",
           "fp64": {"gevals": 2 * n / (ms64 / 1e3) / 1e9, "ms": ms64},
           "fp32_mixed": {"gevals": 2 * n / (ms32 / 1e3) / 1e9, "ms": ms32}}
    regs = {kind: classify(kind, v, x).cpu().numpy() for kind in ("i", "k")}
    res["region_mix"] = {kind: {REGION_NAMES[r]: float(np.mean(regs[kind] == r))
                                for r in range(8) if np.any(regs[kind] == r)} for kind in ("i", "k")}
    if check:
        import oracle
        oracle.build()
        rng = np.random.default_rng(seed + 1)
        err = {"fp64": {}, "fp32_mixed": {}}
        for ki, kind in enumerate(("i", "k")):
            reg = regs[kind]
            for r in range(8):
                sel = np.flatnonzero(reg == r)
                if sel.size == 0:
                    continue
                idx = sel[rng.integers(0, sel.size, min(sel.size, per_region))]
                it = torch.from_numpy(idx).to(dev)
                vs, xs = v[it].cpu().numpy(), x[it].cpu().numpy()
                fn = oracle.log_i if kind == "i" else oracle.log_k
                ref = fn(vs, xs)
                e = oracle.rel_err(out[ki][it].cpu().numpy(), ref, oracle.error_scale(kind, vs, xs))
                err["fp64"]["%s_%s" % (kind, REGION_NAMES[r])] = float(np.max(e))
                vf = vs.astype(np.float32).astype(np.float64)
                xf = xs.astype(np.float32).astype(np.float64)
                ref32 = fn(vf, xf)
                got32 = out32[ki][it].double().cpu().numpy()
                e32 = oracle.rel_err(got32, ref32, oracle.error_scale(kind, vf, xf))
                err["fp32_mixed"]["%s_%s" % (kind, REGION_NAMES[r])] = float(np.max(e32))
        res["max_rel_err_per_region"] = err
        res["samples_per_region"] = per_region
    return res
