"""Throughput on the paper's own test workloads, for context beside its
runtime tables (Sec. 6.1-6.2).

* Fractional orders: the Small region (v, x) ~ U[0, 150]^2 and the Large
  regions [150, 1e4]^2 (log I) and [150, 4000]^2 (log K), 10M uniform pairs
  each (Sec. 5), in the tight dispatch and in the paper's GPU dispatch
  (LB_PAPER_GPU: three expressions, Simpson N = 600 for the K integral).
* Orders 0 and 1: 100M arguments x ~ U[0, 150] (Small) and U[150, 1e4]
  (Large) through the general log I path with a scalar order, beside CUDA's
  cyl_bessel_i0 / cyl_bessel_i1 followed by a log (the paper's comparison
  for these orders; note these overflow to +inf above x ~ 713).
All inputs are generated on the device (seeded Philox) and stay resident;
times are CUDA-event averages over `reps` calls after one warm-up call.
"""
import torch

from paper_2409_08729_gb300 import _binding as B


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


def _uniform(n, lo, hi, g, dev):
    t = torch.empty(n, dtype=torch.float64, device=dev)
    return t.uniform_(lo, hi, generator=g)


def run(device="cuda", n_frac=10_000_000, n_int=100_000_000, reps=3, seed=11):
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    L = B.lib()
    sp = torch.cuda.current_stream(dev).cuda_stream
    res = {"fractional": {}, "orders_0_1": {}}
    regions = {("i", "small"): (0.0, 150.0), ("i", "large"): (150.0, 1e4),
               ("k", "small"): (0.0, 150.0), ("k", "large"): (150.0, 4000.0)}
    out = torch.empty(n_frac, dtype=torch.float64, device=dev)
    for (kind, which), (lo, hi) in regions.items():
        v = _uniform(n_frac, lo, hi, g, dev)
        x = _uniform(n_frac, lo, hi, g, dev)
        fn = L.logbessel_i if kind == "i" else L.logbessel_k
        row = {}
        for mode_name in ("tight", "paper_gpu"):
            mode = B.MODES[mode_name]
            ms = _time(lambda: B.check(fn(B.LB_F64, v.data_ptr(), 1, x.data_ptr(), out.data_ptr(), n_frac, mode,
                                          sp)), reps)
            row[mode_name] = {"ms": ms, "gevals": n_frac / (ms / 1e3) / 1e9}
        res["fractional"]["log_%s_%s" % (kind, which)] = row
        del v, x
    del out
    out = torch.empty(n_int, dtype=torch.float64, device=dev)
    for which, (lo, hi) in (("small", (0.0, 150.0)), ("large", (150.0, 1e4))):
        x = _uniform(n_int, lo, hi, g, dev)
        for order, cuda_fn in ((0, 4), (1, 5)):
            vs = torch.tensor([float(order)], dtype=torch.float64, device=dev)
            ms = _time(lambda: B.check(L.logbessel_i(B.LB_F64, vs.data_ptr(), 0, x.data_ptr(), out.data_ptr(), n_int,
                                                     0, sp)), reps)
            ms_cuda = _time(lambda: B.check(L.logbessel_math_eval(cuda_fn, x.data_ptr(), out.data_ptr(), n_int, sp)),
                            reps)
            res["orders_0_1"]["log_i%d_%s" % (order, which)] = {
                "ms": ms, "gevals": n_int / (ms / 1e3) / 1e9,
                "cuda_cyl_bessel_ms": ms_cuda, "cuda_cyl_bessel_gevals": n_int / (ms_cuda / 1e3) / 1e9}
        del x
    res["sizes"] = {"fractional_pairs": n_frac, "order_0_1_args": n_int}
    return res
