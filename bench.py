"""Benchmark: throughput of log I_v(x) and log K_v(x) on the paper-shaped sweep.

Workload (one step): for each order v in {2^0, ..., 2^10}, 20M arguments
x ~ U[1, 100] (float64), evaluated with one call per order (scalar v) and
once more as a single mixed-order call over all 220M pairs (orders drawn at
random per pair); both log I and log K.  880M evaluations per step, all
through the C ABI in include/logbessel.h.  Inputs are generated on the GPU
(seeded Philox) and stay resident; every call streams >= 160 MB of inputs,
above the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the extended-precision
CPU oracle on the host cores instead (the only reference implementation of
this method available here).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gevals/s (log I_v and log K_v, FP64)"

# DRAM bytes (read + write) per benchmark step of each kernel, from one ncu
# capture of every launch of one full-size step (the launch list of
# profiles/launches_paper_sweep_fp64.md, with dram__bytes_read.sum and
# dram__bytes_write.sum); empty when the kernels changed since.
NCU_DRAM_BYTES_PER_STEP = {"lb_tiles_kernel": (17.417e9, 27), "lb_kint_kernel": (9.431e9, 90)}
# Pipe utilisation of each kernel from ncu --set full on a small case of the
# same workload (profiles/lb_tiles_kernel_sweep_small.md,
# profiles/lb_kint_kernel_sweep_small.md, profiles/fp32_mixed_sweep_small.md):
# share of peak issue of the FP64 pipe, the ALU pipe, the FP32 (FMA) pipe and
# the XU (special-function) pipe while active, and the share of cycles that
# issue; empty when stale.
NCU_PIPES = {
    "lb_tiles_kernel": {"fp64": 0.618, "alu": 0.460, "fma": 0.300, "xu": 0.025, "issue_active": 0.675,
                        "launch": "log I, mixed orders, 11M pairs"},
    "lb_kint_kernel": {"fp64": 0.355, "alu": 0.635, "fma": 0.193, "xu": 0.015, "issue_active": 0.662,
                       "launch": "one-slot class kernel of a mixed-order log K call (class 4: fp64 0.257, "
                                 "alu 0.611, issue 0.634); FMA-heavy pipe (integer multiplies) 0.48; captured "
                                 "before the one-slot rule for orders 0.9-2 was added"},
}
NCU_PIPES_FP32 = {
    "lb_tiles_kernel": {"fp64": 0.0, "alu": 0.450, "fma": 0.235, "xu": 0.111, "issue_active": 0.760,
                        "launch": "log I, mixed orders, 11M pairs"},
    "lb_kint_kernel": {"fp64": 0.0, "alu": 0.518, "fma": 0.312, "xu": 0.054, "issue_active": 0.798,
                       "launch": "log K integral, mixed orders"},
}
UNIT = "Gevals/s"
WORKLOAD = "paper-shaped sweep: v=2^0..2^10 x 20M x~U[1,100] per order, log I + log K, per-order + mixed-order calls"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (ms): the job takes as long as its slowest
    rank.  `dist` is torch.distributed with a process group, or None."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gevals(evals_per_step, steps, world, ms):
    """Whole-job throughput: the evaluations of all ranks (each rank runs the
    same workload: weak scaling) over the slowest rank's time."""
    return evals_per_step * steps * world / (ms / 1e3) / 1e9


def oracle_sample(n_per_v, seed):
    from paper_2409_08729_gb300.workloads import sweep_pairs
    v, x = sweep_pairs(n_per_v, seed=seed)
    return v, x


def time_oracle(n_per_v, seed=7):
    """Oracle throughput (evals/s) over log I and log K on a sample of the sweep."""
    import oracle
    v, x = oracle_sample(n_per_v, seed)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    oracle.log_i(v, x, threads=threads)
    oracle.log_k(v, x, threads=threads)
    dt = time.perf_counter() - t0
    return 2 * v.size / dt, threads, v.size


def reference_arm(args, rank, world):
    """The oracle on the host cores, same metric and workload shape, bounded samples."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    per_v = args.ref_per_v
    for _ in range(args.warmup):
        time_oracle(max(per_v // 10, 10), seed=1)
    rates = []
    t0 = time.perf_counter()
    for s in range(args.steps):
        r, threads, n = time_oracle(per_v, seed=100 + s)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = 2 * per_v * 11 * args.steps / wall / 1e9
    sample = "%d pairs per step (%d per order, log I + log K), drawn from the sweep" % (11 * per_v, per_v)
    # rank 0 alone runs the oracle: the value is that one process's
    # throughput on the host cores, not a whole-job figure over N ranks
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "ranks_used": 1, "value_scope": "rank 0 only (the oracle on the host cores; other ranks idle)",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_per_step": 22 * per_v},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-per-v", type=int, default=20_000_000)
    ap.add_argument("--mode", default="tight", choices=["tight", "paper_gpu"])
    ap.add_argument("--cpu-per-v", type=int, default=20000, help="oracle sample per order for cpu_baseline")
    ap.add_argument("--ref-per-v", type=int, default=4000, help="oracle sample per order per reference step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-dx", action="store_true", help="skip the x-derivative sweep")
    ap.add_argument("--err-sample", type=int, default=4000, help="oracle-checked outputs per call type")
    ap.add_argument("--serve-requests", type=int, default=100_000,
                    help="requests in the serving measurement (0 = skip)")
    ap.add_argument("--serve-per-call-requests", type=int, default=5000,
                    help="requests of the one-call-per-request arm at the offered loads")
    ap.add_argument("--robust-n", type=int, default=64 << 20,
                    help="pairs of the robustness sweep measurement (0 = skip)")
    ap.add_argument("--no-paper-tables", action="store_true",
                    help="skip the paper's Small/Large and order-0/1 workloads")
    args = ap.parse_args()

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import paper_2409_08729_gb300 as lb
    from paper_2409_08729_gb300 import _binding as B
    from benchmarks import optable as OT
    from benchmarks import work as WK
    from paper_2409_08729_gb300.workloads import SWEEP_ORDERS, sweep_device
    lb.build_library()

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    L = B.lib()
    mode = B.MODES[args.mode]
    nv = len(SWEEP_ORDERS)
    n1 = args.n_per_v
    n_all = n1 * nv
    x_all, v_mixed = sweep_device(n1, seed=1234 + rank, device=dev)
    orders = torch.tensor(SWEEP_ORDERS, dtype=torch.float64, device=dev)
    outs = torch.empty((4, n_all), dtype=torch.float64, device=dev)   # I per-order, I mixed, K per-order, K mixed
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step(xa, vm, ob):
        for kind, fn in ((0, L.logbessel_i), (1, L.logbessel_k)):
            o_per, o_mix = ob[2 * kind], ob[2 * kind + 1]
            for k in range(nv):
                B.check(fn(B.LB_F64, orders[k:k + 1].data_ptr(), 0, xa[k * n1:(k + 1) * n1].data_ptr(),
                           o_per[k * n1:(k + 1) * n1].data_ptr(), n1, mode, sp))
            B.check(fn(B.LB_F64, vm.data_ptr(), 1, xa.data_ptr(), o_mix.data_ptr(), n_all, mode, sp))

    evals_per_step = 4 * n_all

    # FP64 rates of this GPU, measured live (the DFMA rate checks the peak
    # derived from unit counts and clock)
    rates = B.measure_fp64(sp)

    for _ in range(args.warmup):
        step(x_all, v_mixed, outs)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs ----
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    B.profile_enable(True)
    launches0 = B.launch_count()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(x_all, v_mixed, outs)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    launches = B.launch_count() - launches0
    prof = B.profile_read()
    B.profile_enable(False)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, pg, dev)
    value = job_gevals(evals_per_step, args.steps, world, ms)

    # ---- end to end: the same step through logbessel_host on pinned host
    # buffers (copy-in, evaluation and copy-out of chunks overlap inside) ----
    e2e = None
    if not args.no_e2e:
        hx = torch.empty(n_all, dtype=torch.float64, pin_memory=True)
        hv = torch.empty(n_all, dtype=torch.float64, pin_memory=True)
        hx.copy_(x_all)
        hv.copy_(v_mixed)
        ho = torch.empty((4, n_all), dtype=torch.float64, pin_memory=True)
        hord = torch.tensor(SWEEP_ORDERS, dtype=torch.float64).pin_memory()

        def step_host():
            for fn in (0, 1):
                o_per, o_mix = ho[2 * fn], ho[2 * fn + 1]
                for k in range(nv):
                    B.check(L.logbessel_host(fn, B.LB_F64, hord[k:k + 1].data_ptr(), 0,
                                             hx[k * n1:(k + 1) * n1].data_ptr(),
                                             o_per[k * n1:(k + 1) * n1].data_ptr(), n1, mode, 0))
                B.check(L.logbessel_host(fn, B.LB_F64, hv.data_ptr(), 1, hx.data_ptr(), o_mix.data_ptr(), n_all,
                                         mode, 0))

        step_host()
        # pinned-copy bandwidth of this machine, both directions, one at a time
        # (the host side varies between boxes; the figure explains the e2e value)
        link = {}
        for name, src, dst in (("h2d_gbs", hx, x_all), ("d2h_gbs", x_all, hx)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            tl = time.perf_counter()
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            link[name] = 3 * n_all * 8 / (time.perf_counter() - tl) / 1e9
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        esampler = ClockSampler(local_rank)
        esampler.start()
        time.sleep(0.3)
        t0h = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        ems = (time.perf_counter() - t0h) * 1e3
        eclocks = esampler.stop()
        ems = max_over_ranks(ems, pg, dev)
        e2e = {"value": job_gevals(evals_per_step, args.steps, world, ems), "unit": UNIT,
               "h2d_bytes_per_step": 2 * (nv * 8 + n1 * 8 * nv + 2 * n_all * 8),
               "d2h_bytes_per_step": 4 * n_all * 8,
               "api": "logbessel_host (C ABI, pinned host buffers, synchronous per call)",
               "pinned_copy_gbs": link, "clocks": eclocks,
               "copy_ms_per_step_at_that_rate": 1e3 * (2 * (nv * 8 + n1 * 8 * nv + 2 * n_all * 8) / link["h2d_gbs"]
                                                       + 4 * n_all * 8 / link["d2h_gbs"]) / 1e9}
        del hx, hv, ho

    # ---- sampled accuracy of the timed outputs (FP64) against the oracle ----
    acc = None
    if rank == 0 and args.err_sample > 0:
        import oracle
        oracle.build()
        rs = np.random.default_rng(5)
        idx = rs.integers(0, n_all, args.err_sample)
        xs = x_all[idx].cpu().numpy()
        vmix = v_mixed[idx].cpu().numpy()
        vper = np.asarray(SWEEP_ORDERS)[idx // n1]
        acc = {}
        for name, row, vv, kind in (("i_per_order", 0, vper, "i"), ("i_mixed", 1, vmix, "i"),
                                    ("k_per_order", 2, vper, "k"), ("k_mixed", 3, vmix, "k")):
            got = outs[row][idx].cpu().numpy()
            ref = oracle.log_i(vv, xs) if kind == "i" else oracle.log_k(vv, xs)
            e = oracle.rel_err(got, ref, oracle.error_scale(kind, vv, xs))
            acc[name] = float(e.max())
        acc["samples_per_call_type"] = int(args.err_sample)

    # ---- the same sweep in the FP32-mixed form ----
    fp32 = None
    if not args.no_fp32:
        x32 = x_all.float()
        v32 = v_mixed.float()
        o32 = torch.empty((4, n_all), dtype=torch.float32, device=dev)
        ord32 = orders.float()

        def step32():
            for kind, fn in ((0, L.logbessel_i), (1, L.logbessel_k)):
                o_per, o_mix = o32[2 * kind], o32[2 * kind + 1]
                for k in range(nv):
                    B.check(fn(B.LB_F32, ord32[k:k + 1].data_ptr(), 0, x32[k * n1:(k + 1) * n1].data_ptr(),
                               o_per[k * n1:(k + 1) * n1].data_ptr(), n1, mode, sp))
                B.check(fn(B.LB_F32, v32.data_ptr(), 1, x32.data_ptr(), o_mix.data_ptr(), n_all, mode, sp))

        for _ in range(2):
            step32()
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        B.profile_enable(True)
        g0.record(stream)
        for _ in range(args.steps):
            step32()
        g1.record(stream)
        torch.cuda.synchronize()
        prof32 = B.profile_read()
        B.profile_enable(False)
        ms32 = max_over_ranks(g0.elapsed_time(g1), pg, dev)
        fp32 = {"value": job_gevals(evals_per_step, args.steps, world, ms32), "unit": UNIT,
                "ms_per_step": ms32 / args.steps, "dtype": "f32 inputs/outputs, FP32-pipe evaluation"}
        if rank == 0 and args.err_sample > 0:
            import oracle
            e_max = 0.0
            for row, vv, kind in ((1, vmix, "i"), (3, vmix, "k")):
                got = o32[row][idx].double().cpu().numpy()
                vf = vv.astype(np.float32).astype(np.float64)
                xf = xs.astype(np.float32).astype(np.float64)
                ref = oracle.log_i(vf, xf) if kind == "i" else oracle.log_k(vf, xf)
                e = oracle.rel_err(got, ref, oracle.error_scale(kind, vf, xf))
                e_max = max(e_max, float(e.max()))
            fp32["max_rel_err_mixed_calls"] = e_max
        del x32, v32, o32

    # ---- the same sweep through the adjoint kernels (d/dx log I, d/dx log K,
    # FP64), with sampled errors against the oracle's Bessel-ratio derivative ----
    dx = None
    if not args.no_dx:
        odx = torch.empty((4, n_all), dtype=torch.float64, device=dev)

        def step_dx():
            for kind, fn in ((0, L.logbessel_i_dx), (1, L.logbessel_k_dx)):
                o_per, o_mix = odx[2 * kind], odx[2 * kind + 1]
                for k in range(nv):
                    B.check(fn(B.LB_F64, orders[k:k + 1].data_ptr(), 0, x_all[k * n1:(k + 1) * n1].data_ptr(),
                               o_per[k * n1:(k + 1) * n1].data_ptr(), n1, mode, sp))
                B.check(fn(B.LB_F64, v_mixed.data_ptr(), 1, x_all.data_ptr(), o_mix.data_ptr(), n_all, mode, sp))

        for _ in range(2):
            step_dx()
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(args.steps):
            step_dx()
        d1.record(stream)
        torch.cuda.synchronize()
        msdx = max_over_ranks(d0.elapsed_time(d1), pg, dev)
        dx = {"value": job_gevals(evals_per_step, args.steps, world, msdx), "unit": UNIT,
              "ms_per_step": msdx / args.steps, "dtype": "f64",
              "calls": "logbessel_i_dx, logbessel_k_dx: the sweep's per-order and mixed-order calls"}
        if rank == 0 and args.err_sample > 0:
            import oracle
            errs = {}
            for name, row, vv, kind in (("i_per_order", 0, vper, "i"), ("i_mixed", 1, vmix, "i"),
                                        ("k_per_order", 2, vper, "k"), ("k_mixed", 3, vmix, "k")):
                got = odx[row][idx].cpu().numpy()
                ref = oracle.dlog_i_dx(vv, xs) if kind == "i" else oracle.dlog_k_dx(vv, xs)
                errs[name] = float((np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)).max())
            dx["max_rel_err"] = errs
        del odx

    # ---- vMF (paper Sec. 6.3): Newton fits of the concentration from the mean
    # resultant length R = A_d(kappa) (the library's own mean ratio, so the fit
    # must return kappa), and the throughput of log C_d and its derivative ----
    vmf = None
    if not args.no_dx:
        from paper_2409_08729_gb300 import vmf as VM
        fits = []
        VM.fit_kappa(2048, 0.5, device=str(dev))   # first call loads the module (untimed)
        for d in (2048, 8192, 32768):
            for kt in (d / 10.0, float(d), 10.0 * d):
                R = float(VM.mean_ratio(d, torch.tensor([kt], dtype=torch.float64, device=dev)))
                torch.cuda.synchronize()
                tf = time.perf_counter()
                res = VM.fit_kappa(d, R, device=str(dev))
                fms = (time.perf_counter() - tf) * 1e3
                fits.append({"d": d, "kappa_true": kt, "R": R, "kappa_hat": res["kappa"],
                             "iterations": res["iterations"], "ms": fms,
                             "rel_dev": abs(res["kappa"] / kt - 1.0)})
        kap = torch.exp(torch.empty(n1, dtype=torch.float64, device=dev).uniform_(np.log(81.92), np.log(819200.0)))
        ov = torch.empty_like(kap)
        rates_vmf = {}
        for name, deriv in (("log_c", 0), ("dlog_c", 1)):
            for _ in range(2):
                B.check(L.logbessel_vmf_log_c(B.LB_F64, 8192.0, kap.data_ptr(), ov.data_ptr(), n1, deriv, sp))
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for _ in range(args.steps):
                B.check(L.logbessel_vmf_log_c(B.LB_F64, 8192.0, kap.data_ptr(), ov.data_ptr(), n1, deriv, sp))
            v1.record(stream)
            torch.cuda.synchronize()
            rates_vmf[name + "_gevals"] = n1 * args.steps / (v0.elapsed_time(v1) * 1e-3) / 1e9
        vmf = {"fits": fits, "max_rel_dev": max(f["rel_dev"] for f in fits),
               "throughput": dict(rates_vmf, d=8192, n=n1, kappa="log-uniform [d/100, 100 d]")}
        del kap, ov

    # ---- rooflines: algorithmic work of one step from the fixed operation
    # table (benchmarks/optable.py), per kernel, over the CUDA-event time of
    # the kernel's launches in the timed region ----
    wk = {}
    for kind in ("i", "k"):
        for k in range(nv):
            WK.merge(wk, WK.call_work(kind, orders[k:k + 1], x_all[k * n1:(k + 1) * n1], seed=k))
        WK.merge(wk, WK.call_work(kind, v_mixed, x_all, seed=100))
    kern_ops = {"lb_tiles_kernel": WK.ops_of(wk, "tiles"), "lb_kint_kernel": WK.ops_of(wk, "kint")}
    fb_pairs = sum(c for c, _ in wk["kint"].values())
    # algorithmic bytes per step: per pair x (and v when one per pair) read
    # and the result written (8 B each); K-integral pairs: the tile kernel
    # writes a 4 B queue entry, the K-integral kernel reads the entry, v and
    # x and writes the result
    alg_bytes = {"lb_tiles_kernel": 2 * (nv * n1 * 16 + n_all * 24) - fb_pairs * 4,
                 "lb_kint_kernel": fb_pairs * 4 + fb_pairs * 20}
    kernels = {}
    for kname, ops in kern_ops.items():
        nl, ntimed, kms = prof.get(kname, (0, 0, 0.0))
        if not ntimed or kms <= 0:
            continue
        ach = ops * args.steps / (kms / 1e3)
        traffic = NCU_DRAM_BYTES_PER_STEP.get(kname)
        kernels[kname] = {"launches": ntimed, "ms": kms, "avg_launch_ms": kms / ntimed,
                          "ops_per_step": ops, "achieved": ach / 1e9, "frac": ach / OT.PEAK_FP64_OPS,
                          "algorithmic_bytes_per_launch": alg_bytes[kname] * args.steps / ntimed,
                          "traffic": traffic[0] * args.steps / ntimed if traffic else None,
                          "ncu": NCU_PIPES.get(kname)}
    name = max(kernels, key=lambda k: kernels[k]["ms"])
    kd = kernels[name]
    roof = {"bound": "alu", "kernel": name, "achieved": kd["achieved"], "peak": OT.PEAK_FP64_OPS / 1e9,
            "unit": "G FP64 op/s", "frac": kd["frac"], "traffic": kd["traffic"],
            "algorithmic_bytes": kd["algorithmic_bytes_per_launch"], "launches": kd["launches"],
            "avg_launch_ms": kd["avg_launch_ms"],
            "work": "FP64 operations of the method (benchmarks/optable.py) at per-pair term and node counts; "
                    "library calls (log, exp, rcp, rsqrt, lgamma) not priced; the high-order terms of the "
                    "mu_20 and U_K sums execute as double-float FP32 instructions, so the rate counts the "
                    "method's operations, not the FP64 instructions issued",
            "peak_source": "152 SMs x 2 FP64 op/clk x 2.07 GHz; live DFMA microbenchmark %.1f G/s"
                           % (rates["dfma"] / 1e9),
            "ncu": kd["ncu"]}
    work_by_region = {kern: {r: {"pairs": c, "ops_per_pair": m} for r, (c, m) in regs.items()}
                      for kern, regs in wk.items()}
    if fp32 is not None:
        wk32 = {}
        x32 = x_all.float()
        v32 = v_mixed.float()
        ord32 = orders.float()
        for kind in ("i", "k"):
            for k in range(nv):
                WK.merge(wk32, WK.call_work(kind, ord32[k:k + 1], x32[k * n1:(k + 1) * n1], fp32=True, seed=k))
            WK.merge(wk32, WK.call_work(kind, v32, x32, fp32=True, seed=100))
        del x32, v32
        k32 = {}
        for kname, kern in (("lb_tiles_kernel", "tiles"), ("lb_kint_kernel", "kint")):
            nl, ntimed, kms = prof32.get(kname, (0, 0, 0.0))
            if not ntimed or kms <= 0:
                continue
            ops = WK.ops_of(wk32, kern)
            ach = ops * args.steps / (kms / 1e3)
            k32[kname] = {"launches": ntimed, "ms": kms, "ops_per_step": ops, "achieved": ach / 1e9,
                          "frac_fp32_pipe": ach / OT.PEAK_FP32_OPS, "ncu": NCU_PIPES_FP32.get(kname)}
        n32 = max(k32, key=lambda k: k32[k]["ms"])
        fp32["roofline"] = {"bound": "alu", "kernel": n32, "achieved": k32[n32]["achieved"],
                            "peak": OT.PEAK_FP32_OPS / 1e9, "unit": "G FP32 op/s",
                            "frac": k32[n32]["frac_fp32_pipe"], "traffic": None,
                            "peak_source": "152 SMs x 128 FP32 op/clk x 2.07 GHz",
                            "fp64_pipe": "no FP64 operations on this path (FP32 everywhere)",
                            "bound_by": "instruction issue (ncu issue active %.2f; FP32 pipe %.2f)"
                                        % (NCU_PIPES_FP32[n32]["issue_active"], NCU_PIPES_FP32[n32]["fma"])
                                        if n32 in NCU_PIPES_FP32 else None,
                            "ncu": NCU_PIPES_FP32.get(n32)}
        fp32["kernels"] = k32
        fp32["work_by_region"] = {kern: {r: {"pairs": c, "ops_per_pair": m} for r, (c, m) in regs.items()}
                                  for kern, regs in wk32.items()}
    mix = {}
    for nm, (c, _) in wk["tiles"].items():
        mix[nm] = c / (4 * n_all)
    mix["k_integral"] = fb_pairs / (4 * n_all)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "evals_per_step": evals_per_step, "n_per_order": n1,
                       "mode": args.mode, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (>=160 MB per call), no flush"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clocks,
            "kernels": kernels, "work_by_region": work_by_region, "region_mix_step": mix,
            "fp64_rates": {k: v / 1e9 for k, v in rates.items()}}
    line["max_rel_err"] = acc
    line["fp32_mixed"] = fp32
    line["derivatives"] = dx
    line["vmf"] = vmf
    del outs
    torch.cuda.empty_cache()
    if rank == 0 and args.robust_n > 0:
        from benchmarks import robustbench
        line["robustness_sweep"] = robustbench.run(n=args.robust_n, device=str(dev),
                                                   per_region=1000 if args.err_sample > 0 else 0,
                                                   check=args.err_sample > 0)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_paper_tables:
        from benchmarks import paperbench
        line["paper_workloads"] = paperbench.run(device=str(dev))
        torch.cuda.empty_cache()
    if rank == 0 and args.serve_requests > 0:
        from benchmarks import servebench
        line["serving"] = servebench.run(n_req=args.serve_requests, seed=0, device=str(dev),
                                         load=[0.5, 0.8, 0.95], per_call_requests=args.serve_per_call_requests)
    if rank == 0:
        r, threads, n = time_oracle(args.cpu_per_v)
        line["cpu_baseline"] = {"value": r / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "%d pairs of the sweep (%d per order), log I + log K" % (n, args.cpu_per_v)}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
