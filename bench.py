"""Benchmark: st-HOSVD-ALS time-to-tolerance on the 512^3 FP32 workload.

Workload: 512 x 512 x 512 FP32 tensor (512 MiB) of multilinear rank (32,32,32)
with a 1/k core spectrum, Haar factors and 1e-2 relative Gaussian noise;
st-HOSVD-ALS to eta = 1e-6 (at most 50 sweeps per mode). One step = one full
decomposition (all modes: initial guess, ALS sweeps until the stop rule, the
truncations) -- one graph launch through the C ABI. The input (512 MiB) is
larger than L2, so no flush is needed between steps.

The timed path is the mixed-precision one (BF16 tensor-core bulk sweeps, FP32
finishing sweeps, FP64 small algebra); the plain FP32 path is timed in the same
run and reported beside it with both errors ("mixed vs FP32 plain at equal
error"). --precision native makes the plain path the timed one.

Prints one JSON line (see the keys below). Under torchrun each rank runs an
independent replica on its own GPU (weak scaling, no collective on the data
path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "st-HOSVD-ALS time-to-tol & HBM GB/s (% peak), mixed vs FP32 plain at equal error"
# DRAM bytes (read + write) per launch on the 512^3 mode-1 view, from ncu captures of
# the 512x512x256 case scaled by 2 (traffic grows with the columns processed); None
# where no capture of the current kernel exists.
PASS_TRAFFIC = 2 * (268599552 + 14900480)   # CUDA-core FP32 fused pass
TC_TRAFFIC = 2 * (134338048 + 3646208)      # BF16 tensor-core fused pass
T32_TRAFFIC = {"w": 2 * (268631040 + 12190976),   # split-precision W and Y passes
               "y": 2 * (285368320 + 3259648)}
PROD_TRAFFIC = {"w": 2 * (268647424 + 8675840),    # two-product form: register-tiled W product
                "y": 2 * (285284096 + 6981632)}    # and the split-K Y = B W kernel
DIMS = (512, 512, 512)
RANKS = (32, 32, 32)
ETA = 1e-6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _job_ms(ms, dist, device="cuda"):
    """Time of one weak-scaled step of the whole job: every rank times its own
    replica, and the step lasts as long as the slowest rank (max over ranks),
    followed by a barrier. Single process: the rank's own time."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def _job_value(world, ms, units_per_rank=1.0):
    """Whole-job throughput: the units every rank processed in one step, per second
    of the slowest rank's step time."""
    return world * units_per_rank * 1e3 / ms


def _cpu_oracle_run(a64, ranks, eta):
    from oracle import tucker_oracle as O
    t0 = time.perf_counter()
    res = O.st_hosvd_als(a64, ranks, eta=eta, seed=1)
    return time.perf_counter() - t0, res


def _full_input():
    """The benchmark's 512^3 input (the GPU arm's seed and recipe), as FP64."""
    import numpy as np
    import workloads as W
    cfg = W.CONFIGS["c512_f32"]
    p = W.planted(cfg.seed, DIMS, RANKS, cfg.core, cfg.noise_rel, dtype=np.float32)
    return p.A.astype(np.float64)


def _cpu_sample(budget_s: float = 10.0):
    """The oracle, as it stands, on the full 512^3 workload, repeated until about
    budget_s of host time has been spent (at least once)."""
    cores = len(os.sched_getaffinity(0))
    a64 = _full_input()
    times = []
    while not times or sum(times) < budget_s:
        dt, _ = _cpu_oracle_run(a64, RANKS, ETA)
        times.append(dt)
    t = sum(times) / len(times)
    return {"value": 1.0 / t, "unit": "st-HOSVD/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 NumPy oracle st-HOSVD-ALS on the full 512x512x512 input, "
                      f"{len(times)} runs of {t:.2f} s",
            "seconds": t}


def run_reference(args):
    """The oracle as the reference arm: the full 512^3 st-HOSVD-ALS per step on the
    host cores (the GPU arm's input, seed and tolerance)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    a64 = _full_input()
    for _ in range(args.warmup):
        _cpu_oracle_run(a64, RANKS, ETA)
    times = []
    for _ in range(args.steps):
        dt, _ = _cpu_oracle_run(a64, RANKS, ETA)
        times.append(dt)
    t = sum(times) / len(times)
    value = 1.0 / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "st-HOSVD/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "st-HOSVD-ALS 512x512x512 FP32 rank (32,32,32) 1/k spectrum "
                                   "1e-2 noise eta 1e-6"},
            "cpu_baseline": {"value": value, "unit": "st-HOSVD/s", "cores": cores, "kind": "oracle",
                             "sample": "FP64 NumPy oracle on the full 512x512x512 input per step"},
            "e2e": {"value": value, "unit": "st-HOSVD/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tals", choices=["tals", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed_bf16", choices=["native", "mixed_bf16"])
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--dims", default=None, help="override tensor sizes (profiling), e.g. 512,512,256")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven sweep loop instead of the CUDA graph (same kernels; ncu "
                         "cannot profile kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the other precision path (per-path launch lists under ncu)")
    ap.add_argument("--profile-pass", action="store_true",
                    help="only launch the mode-1 sweep pass twice (for an ncu capture)")
    ap.add_argument("--profile-what", default="pass", choices=["pass", "tf32", "products", "decomp"],
                    help="with --profile-pass: pass (the fused sweep pass), tf32 (the split-precision "
                         "W and Y passes, one timed launch each after one warm-up), products (the "
                         "two-product form's mode product and split-K Y product, likewise), decomp "
                         "(one decomposition: its split sweep's W product and W statistics)")
    ap.add_argument("--batch-count", type=int, default=4096,
                    help="c4: number of tensors (4096 is the workload; fewer for profiling)")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "tucker", "rank500"],
                    help="c2 (default): 512^3 FP32 st-HOSVD, the benchmark line; c1: 64^3 FP64; "
                         "c3: 128^4 FP32 mixed vs plain; c4: 4096 small tensors batched vs "
                         "per-tensor loop; c5: 1024x1024x512 forward + reconstruction-loss backward; "
                         "tucker: the Sec. 6.1.2 Tucker model; rank500: the Sec. 6.4 dense test")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c2":
        from_extra = {"c1": run_c1, "c3": run_c3, "c4": run_c4, "c5": run_c5,
                      "tucker": run_tucker, "rank500": run_rank500}[args.workload]
        return from_extra(args)
    global DIMS
    if args.dims:
        DIMS = tuple(int(x) for x in args.dims.split(","))

    import numpy as np
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    import paper_2004_02583_gb300 as tals
    import workloads as W

    cfg = W.CONFIGS["c512_f32"]
    p = W.planted(cfg.seed, DIMS, RANKS, cfg.core, cfg.noise_rel, dtype=np.float32)
    A = torch.from_numpy(p.A).cuda()
    stream = torch.cuda.current_stream()
    ctx = tals.Context(A, RANKS, eta=ETA, seed=1, precision=args.precision,
                       use_graph=not args.no_graph)
    if args.profile_pass:
        if args.profile_what in ("tf32", "products"):
            ms_, by_, fl_ = ctx.time_sweep(mode=0, engine=args.profile_what, iters=1)
        elif args.profile_what == "decomp":
            G = torch.empty(RANKS, device="cuda")
            Us = [torch.empty((d, r), device="cuda") for d, r in zip(DIMS, RANKS)]
            _, _, st_ = ctx.st_hosvd(G, Us)
            ms_, by_, fl_ = None, None, None
            print(json.dumps({"sweeps": st_["sweeps"], "split_sweeps": st_["split_sweeps"]}))
        else:
            ms_, by_, fl_ = ctx.time_pass(mode=0, iters=1)
        print(json.dumps({"profile_pass_ms": ms_, "bytes": by_, "flops": fl_}))
        ctx.close()
        return
    G = torch.empty(RANKS, device="cuda")
    Us = [torch.empty((d, r), device="cuda") for d, r in zip(DIMS, RANKS)]

    for _ in range(max(3, args.warmup)):
        _, _, st = ctx.st_hosvd(G, Us)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sweeps_total = 0
    for _ in range(args.steps):
        _, _, st = ctx.st_hosvd(G, Us)
        sweeps_total += sum(st["sweeps"])
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = _job_ms(ev0.elapsed_time(ev1) / args.steps, dist)
    clk = clocks.stop() if rank == 0 else {}

    # the other precision path on the same input, for the equal-error comparison
    if args.no_compare:
        ctx.close()
        print(json.dumps({"precision": args.precision, "ms_per_step": ms, "sweeps": st["sweeps"]}))
        return
    other = "native" if args.precision == "mixed_bf16" else "mixed_bf16"
    octx = tals.Context(A, RANKS, eta=ETA, seed=1, precision=other, use_graph=not args.no_graph)
    for _ in range(3):
        octx.st_hosvd(G, Us)
    torch.cuda.synchronize()
    oev0 = torch.cuda.Event(enable_timing=True)
    oev1 = torch.cuda.Event(enable_timing=True)
    oev0.record(stream)
    for _ in range(args.steps):
        _, _, ost = octx.st_hosvd(G, Us)
    oev1.record(stream)
    torch.cuda.synchronize()
    o_ms = oev0.elapsed_time(oev1) / args.steps
    nctx = ctx if args.precision == "native" else octx
    mctx = ctx if args.precision == "mixed_bf16" else octx

    def timed(fn, n):
        for _ in range(2):
            out = fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n, out

    # the plain FP32 path with its products on the CUDA cores (exact FP32 FMA), the
    # previous form of the plain path
    cctx = tals.Context(A, RANKS, eta=ETA, seed=1, precision="native", fp32_engine="cuda",
                        use_graph=not args.no_graph)
    cuda_ms, (_, _, cst) = timed(lambda: cctx.st_hosvd(G, Us), max(3, args.steps // 2))
    # t-HOSVD-ALS (Alg. 4) on the same input, both precision paths
    t_ms, t_rel = {}, {}
    for name, c in (("fp32_plain", nctx), ("mixed", mctx)):
        t_ms[name], (_, _, tst) = timed(lambda: c.t_hosvd(G, Us), max(3, args.steps // 2))
        t_rel[name] = tst["rel_err"]
    # re-run the timed path once so G and U hold its result
    _, _, st = ctx.st_hosvd(G, Us)

    # dominant kernels: the split-precision passes of the FP32 sweeps (W pass, then the
    # Y pass with the residual) over the full tensor (mode-1 view), timed with CUDA
    # events on the stream they are launched on, in the configuration of the step
    mode0 = st["order"][0]
    t32_ms, t32_bytes, t32_flops = nctx.time_sweep(mode=mode0, engine="tf32", iters=10)
    # the exact-FP32 CUDA-core fused pass and the BF16 tensor-core pass, same view
    pass_ms, pass_bytes, pass_flops = nctx.time_pass(mode=mode0, iters=5)
    tc_ms, tc_bytes, tc_flops = mctx.time_pass(mode=mode0, iters=10)
    # the two-product form the FP32 sweeps of the first mode run on in both paths:
    # the register-tiled W product and the split-K Y kernel, each timed alone
    pr_ms, pr_bytes, pr_flops = nctx.time_sweep(mode=mode0, engine="products", iters=10)
    octx_close = octx.close
    cctx.close()
    # the metric's own mixed-vs-plain comparison at equal error on the 128^4 workload
    c3cfg = W.CONFIGS["q128_f32"]
    A3 = torch.from_numpy(W.make(c3cfg).A).cuda()
    G3 = torch.empty(c3cfg.ranks, device="cuda")
    U3 = [torch.empty((d, r), device="cuda") for d, r in zip(c3cfg.dims, c3cfg.ranks)]
    c3 = {}
    for prec in ("mixed_bf16", "native"):
        c = tals.Context(A3, c3cfg.ranks, eta=c3cfg.eta, seed=1, precision=prec,
                         use_graph=not args.no_graph)
        c3[prec] = timed(lambda: c.st_hosvd(G3, U3), max(3, args.steps // 2))
        c.close()
    del A3
    # the CP-model workload of Sec. 6.1.1 at its largest size: 100 x 100 x 10000 FP32,
    # truncation (20, 20, 20), lambda_r in [5, 10], absolute noise 1e-4 (400 MB, larger
    # than L2); the third mode (10000) runs the two-pass sweep
    cpm = W.cp_model(W.CP_SEED, 100, dtype=np.float32)
    Acp = torch.from_numpy(cpm.A).cuda()
    rcp = (20, 20, 20)
    Gcp = torch.empty(rcp, device="cuda")
    Ucp = [torch.empty((d, 20), device="cuda") for d in cpm.A.shape]
    cp = {}
    for drv in ("st", "t"):
        c = tals.Context(Acp, rcp, eta=1e-4, seed=1, use_graph=not args.no_graph)
        fn = (lambda: c.st_hosvd(Gcp, Ucp)) if drv == "st" else (lambda: c.t_hosvd(Gcp, Ucp))
        cp[drv] = timed(fn, max(3, args.steps // 2))
        c.close()
    del Acp, cpm
    # HOOI refinement (Sec. 6.3) started from the 512^3 st-HOSVD-ALS factors, FP32,
    # stop at a residual change below 1e-5 (FP32 resolves r to about 1e-5 here)
    Uh = [u.clone() for u in Us]
    Gh = torch.empty(RANKS, device="cuda")

    def run_hooi():
        V = [u.clone() for u in Uh]
        return nctx.hooi(V, G=Gh, tol=1e-5, max_iters=10, inner_eta=1e-9, inner_sweeps=10)
    hooi_ms, (_, _, hinfo) = timed(run_hooi, 3)

    # end to end through the C ABI with host buffers (H2D of A, D2H of G and U)
    e_ms, e_single_ms, h2d, d2h = None, None, 0, 0
    if not args.no_e2e:
        hctx = tals.HostContext(DIMS, RANKS, "f32", eta=ETA, seed=1, precision=args.precision)
        A_h = torch.from_numpy(p.A).pin_memory()
        G_h = torch.empty(RANKS).pin_memory()
        U_h = [torch.empty((d, r)).pin_memory() for d, r in zip(DIMS, RANKS)]
        for _ in range(2):
            hctx.st_hosvd(A_h, G_h, U_h)
        torch.cuda.synchronize()
        # one call per tensor: upload, decomposition, download, nothing overlapped
        e0 = time.perf_counter()
        e_steps = max(3, args.steps // 2)
        for _ in range(e_steps):
            hctx.st_hosvd(A_h, G_h, U_h)
        e_single_ms = (time.perf_counter() - e0) * 1e3 / e_steps
        # pipelined over a stream of tensors (st_hosvd_host_many): every step uploads its
        # full tensor and downloads its core and factors; the upload of step k+1 runs
        # while step k is decomposed (the first upload is not hidden and is included)
        p_steps = max(3, args.steps)
        hctx.st_hosvd_many([A_h] * 2, [G_h] * 2, [U_h] * 2)   # both buffers' graphs built
        e0 = time.perf_counter()
        hctx.st_hosvd_many([A_h] * p_steps, [G_h] * p_steps, [U_h] * p_steps)
        e_ms = (time.perf_counter() - e0) * 1e3 / p_steps
        h2d = A_h.numel() * 4
        d2h = G_h.numel() * 4 + sum(u.numel() * 4 for u in U_h)
        hctx.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, peak_kind = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # split-precision passes (HBM roofline): the dominant one is the headline roofline
    names = {"w": "tals::t32_wpass_kernel<32> (split-precision W = B^T Q on tcgen05 kind::tf32)",
             "y": "tals::t32_ypass_kernel<32> (split-precision Y = B W and the residual "
                  "||B - Q W^T||^2 on tcgen05 kind::tf32)"}
    passes = {}
    for k, i in (("w", 0), ("y", 1)):
        gbs = t32_bytes[i] / (t32_ms[i] * 1e-3) / 1e9
        passes[k] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(gbs / hbm, 4), "traffic": T32_TRAFFIC[k], "kernel": names[k],
                     "algorithmic_bytes": t32_bytes[i], "pass_ms": round(t32_ms[i], 4)}
    # the split-precision engine (fp32_engine = "tensor"; not on the default path)
    dom = "y" if t32_ms[1] >= t32_ms[0] else "w"
    roofline_tf32 = dict(passes[dom])
    roofline_tf32["peak_source"] = f"HBM {hbm} GB/s ({peak_kind}; the pass is timed alone)"
    sweep_ms = t32_ms[0] + t32_ms[1]
    roofline_tf32["sweep"] = {"ms": round(sweep_ms, 4),
                              "gbs": round((t32_bytes[0] + t32_bytes[1]) / (sweep_ms * 1e-3) / 1e9, 1),
                              "fp32_equivalent_tflops": round(t32_flops / (sweep_ms * 1e-3) / 1e12, 2),
                              "other_pass": passes["w" if dom == "y" else "y"]}
    achieved_gbs = pass_bytes / (pass_ms * 1e-3) / 1e9
    achieved_tflops = pass_flops / (pass_ms * 1e-3) / 1e12
    # CUDA-core pass: 152 SMs x 128 FP32 FMA x 2 flops x SM clock (an ALU roofline)
    alu_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    roofline_cuda = {
        "bound": "alu", "achieved": round(achieved_tflops, 2), "peak": round(alu_peak, 2),
        "unit": "TFLOP/s", "frac": round(achieved_tflops / alu_peak, 4), "traffic": PASS_TRAFFIC,
        "kernel": "tals::pass_kernel<float,32,4,16,256> (exact-FP32 CUDA-core fused sweep: the later "
                  "modes' sweeps, and every FP32 sweep with fp32_engine = cuda)",
        "view": "mode-1 view 1 x 512 x 262144, rank 32",
        "algorithmic_bytes": pass_bytes, "algorithmic_flops": pass_flops,
        "hbm_gbs_achieved": round(achieved_gbs, 1), "hbm_frac": round(achieved_gbs / hbm, 4),
        "pass_ms": round(pass_ms, 4),
        "peak_source": f"FP32 FMA peak from {sms} SMs x 128 lanes x 2 flops x median SM clock "
                       f"{sm_mhz} MHz (derived)",
    }
    # the two-product form: each product 2 T R flops over T (+ W) elements
    prod = {}
    pnames = {"w": "tals::mg_pipe<0,0,0,32> (register-tiled mode product W = B x_1 Q^T of the "
                   "two-product FP32 sweep)",
              "y": "tals::adjoint_rows_kernel<32> (split-K Y = B_(1) W of the two-product FP32 sweep)"}
    for k, i in (("w", 0), ("y", 1)):
        tf = pr_flops / 2.0 / (pr_ms[i] * 1e-3) / 1e12
        prod[k] = {"bound": "alu", "achieved": round(tf, 2), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                   "frac": round(tf / alu_peak, 4), "traffic": PROD_TRAFFIC[k], "kernel": pnames[k],
                   "algorithmic_flops": pr_flops / 2.0, "algorithmic_bytes": pr_bytes[i],
                   "hbm_gbs_achieved": round(pr_bytes[i] / (pr_ms[i] * 1e-3) / 1e9, 1),
                   "pass_ms": round(pr_ms[i], 4),
                   "peak_source": f"FP32 FMA peak from {sms} SMs x 128 lanes x 2 flops x median SM clock "
                                  f"{sm_mhz} MHz (derived)"}
    roofline = dict(prod["w"])
    roofline["kernel"] += ("; the largest share among the step's product kernels in both paths (the "
                           "R x R small algebra, a chain of latency-bound one-CTA kernels, is 43% of "
                           "the mixed launch list, small_kernel alone 20%)")
    roofline["view"] = "mode-1 view 1 x 512 x 262144, rank 32"
    tc_gbs = tc_bytes / (tc_ms * 1e-3) / 1e9
    tc_tflops = tc_flops / (tc_ms * 1e-3) / 1e12
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    roofline_tc = {
        "bound": "hbm", "achieved": round(tc_gbs, 1), "peak": hbm, "unit": "GB/s",
        "frac": round(tc_gbs / hbm, 4), "traffic": TC_TRAFFIC,
        "kernel": "tals::tc_pass_kernel<32> (tcgen05 BF16 sweep of the mixed path's bulk sweeps, "
                  "same view)",
        "algorithmic_bytes": tc_bytes, "pass_ms": round(tc_ms, 4),
        "tensor_tflops_achieved": round(tc_tflops, 2),
        "tensor_frac": round(tc_tflops / bf16_peak, 4),
        "peak_source": f"HBM {hbm} GB/s ({peak_kind}); dense BF16 burst {bf16_peak} TFLOP/s ({peak_kind})",
    }
    # kernels per step: per mode 10 (initial guess chain) + the factor copy, 9 per
    # CUDA-core or BF16 sweep, 12 per split-precision sweep (basis split, W pass,
    # ||W||^2 sum, Y pass + the 8-kernel tail), 10 per FP32 sweep on the two-product
    # form (mode product, split-K Y product + the tail); per FP32 sweep of a mode whose
    # sweeps can run split, 4 more on the fused pass (W product, W statistics, test,
    # Y pass) or 2 more on the two-product form (W statistics, test), each exiting at
    # once when its sweep is not split; plus the BF16 conversion of each mode that
    # runs bulk sweeps
    def _extra(prod, sc):
        return (1 + (2 if sc else 0)) if prod else (4 if sc else 0)

    launches = (sum(11 + 9 * n + 3 * t + (n - b) * _extra(pr, sc)
                    for n, t, b, sc, pr in zip(st["sweeps"], st["tc_sweeps"], st["bulk_sweeps"],
                                               st["split_capable"], st["two_product"])) +
                sum(1 for b in st["bulk_sweeps"] if b > 0))
    mixed_st = st if args.precision == "mixed_bf16" else ost
    plain_st = st if args.precision == "native" else ost
    mixed_ms = ms if args.precision == "mixed_bf16" else o_ms
    plain_ms = ms if args.precision == "native" else o_ms
    value = _job_value(world, ms)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "st-HOSVD/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "native" else "bf16+f32", "data": "synthetic",
        "config": {"workload": "st-HOSVD-ALS 512x512x512 FP32 rank (32,32,32) 1/k spectrum "
                               "1e-2 noise eta 1e-6", "precision": args.precision,
                   "time_to_tol_ms": round(ms, 4), "sweeps": st["sweeps"],
                   "split_sweeps": st["split_sweeps"], "two_product": st["two_product"],
                   "bulk_sweeps": st["bulk_sweeps"], "tc_sweeps": st["tc_sweeps"],
                   "rel_err": st["rel_err"],
                   "mixed_vs_fp32_plain": {
                       "mixed_ms": round(mixed_ms, 4), "fp32_plain_ms": round(plain_ms, 4),
                       "speedup": round(plain_ms / mixed_ms, 3),
                       "mixed_rel_err": mixed_st["rel_err"], "fp32_plain_rel_err": plain_st["rel_err"],
                       "rel_err_gap": abs(mixed_st["rel_err"] - plain_st["rel_err"]),
                       "fp32_plain_sweeps": plain_st["sweeps"],
                       "fp32_plain_products": "exact FP32 on the CUDA cores (fused sweep; a sweep "
                                               "predicted to be the last forms W alone first)",
                       "fp32_cuda_core_ms": round(cuda_ms, 4), "fp32_cuda_core_rel_err": cst["rel_err"],
                       "fp32_cuda_core_sweeps": cst["sweeps"]},
                   "c3_128quartic": {
                       "workload": "st-HOSVD-ALS 128^4 FP32 rank (16,16,16,16) 0.8^k spectrum 1e-3 "
                                   "noise eta 1e-6",
                       "mixed_ms": round(c3["mixed_bf16"][0], 4), "fp32_plain_ms": round(c3["native"][0], 4),
                       "speedup": round(c3["native"][0] / c3["mixed_bf16"][0], 3),
                       "mixed_rel_err": c3["mixed_bf16"][1][2]["rel_err"],
                       "fp32_plain_rel_err": c3["native"][1][2]["rel_err"],
                       "rel_err_gap": abs(c3["mixed_bf16"][1][2]["rel_err"] - c3["native"][1][2]["rel_err"]),
                       "mixed_sweeps": c3["mixed_bf16"][1][2]["sweeps"],
                       "fp32_plain_sweeps": c3["native"][1][2]["sweeps"]},
                   "cp_model_100": {
                       "workload": "CP model (Sec. 6.1.1) 100x100x10000 FP32, 20 terms, lambda in "
                                   "[5,10], noise 1e-4, truncation (20,20,20), eta 1e-4",
                       "st_hosvd_ms": round(cp["st"][0], 4), "t_hosvd_ms": round(cp["t"][0], 4),
                       "st_rel_err": cp["st"][1][2]["rel_err"], "t_rel_err": cp["t"][1][2]["rel_err"],
                       "st_sweeps": cp["st"][1][2]["sweeps"], "t_sweeps": cp["t"][1][2]["sweeps"]},
                   "hooi": {"workload": "HOOI (Sec. 6.3) from the 512^3 st-HOSVD-ALS factors, FP32, "
                                       "tol 1e-5, inner ALS eta 1e-9",
                            "ms": round(hooi_ms, 4), "cycles": hinfo["iters"],
                            "resid0": hinfo["resid"][0], "resid": hinfo["resid"][-1],
                            "inner_sweeps": hinfo["inner_sweeps"]},
                   "t_hosvd": {"fp32_plain_ms": round(t_ms["fp32_plain"], 4),
                               "mixed_ms": round(t_ms["mixed"], 4),
                               "fp32_plain_rel_err": t_rel["fp32_plain"], "mixed_rel_err": t_rel["mixed"]},
                   "l2": "inputs (512 MiB) larger than L2",
                   "driver": "host loop" if args.no_graph else "CUDA graph with device-side while",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "roofline_adjoint": prod["y"],
        "roofline_fused": roofline_cuda,
        "roofline_tc": roofline_tc,
        "roofline_tf32": roofline_tf32,
        "e2e": None if e_ms is None else
               {"value": round(world * 1e3 / e_ms, 3), "unit": "st-HOSVD/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e_ms, 3),
                "api": "st_hosvd_host_many (pinned host buffers; the upload of step k+1 overlaps "
                       "step k's decomposition; host-to-device link ~211 GB/s on this box)",
                "single_call_ms_per_step": round(e_single_ms, 3)},
        "gpu_launches": launches * args.steps,
        "launches_per_step": launches,
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                   "reasons": clk.get("reasons", [])},
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = _cpu_sample()
    print(json.dumps(line), flush=True)
    octx_close()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# The other configurations (parity cases of the test suite), measured the same
# way: CUDA events on the launching stream, >= 3 warm-up runs, an L2 flush
# between runs whose inputs fit in L2, the oracle timed on the host beside it.
# ---------------------------------------------------------------------------

def _clock_line(clk):
    return {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
            "reasons": clk.get("reasons", [])}


def _time_gpu(fn, steps, warmup, flush_bytes=0):
    """Mean ms of fn() over `steps` runs, each bracketed by CUDA events; with
    flush_bytes > 0 a buffer that large is written before every run (outside
    the events) so no input stays in L2."""
    import torch
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda") if flush_bytes else None
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    tot, out = 0.0, None
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps, out


def _oracle_time(fn, budget_s=10.0):
    """Repeat the oracle call until about budget_s has passed; mean seconds."""
    t0 = time.perf_counter()
    n = 0
    while True:
        fn()
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el / n * (n + 1) > 3 * budget_s:
            return el / n, n


def _alu_peaks(sms, sm_mhz):
    # FP32: 128 FMA lanes per SM; FP64: the nominal 1.25 TFLOP/s of the part,
    # scaled to the observed clock (the max SM clock is 2070 MHz)
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12, 1.25 * sm_mhz / 2070.0


def run_c1(args):
    """64^3 FP64 st-HOSVD-ALS, rank (8,8,8), eta 1e-8."""
    import numpy as np
    import torch
    import paper_2004_02583_gb300 as tals
    import workloads as W
    from oracle import tucker_oracle as O
    cfg = W.CONFIGS["st64_f64"]
    p = W.make(cfg)
    A = torch.from_numpy(p.A).cuda()
    ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision="native")
    G = torch.empty(cfg.ranks, dtype=torch.float64, device="cuda")
    Us = [torch.empty((d, r), dtype=torch.float64, device="cuda") for d, r in zip(cfg.dims, cfg.ranks)]
    clocks = Clocks(0)
    clocks.start()
    ms, (_, _, st) = _time_gpu(lambda: ctx.st_hosvd(G, Us), args.steps, args.warmup, 256 << 20)
    clk = clocks.stop()
    pass_ms, by, fl = ctx.time_pass(mode=st["order"][0], iters=20)
    ref = O.st_hosvd_als(p.A, cfg.ranks, eta=cfg.eta, seed=1)
    rel_own = O.rel_error(p.A, G.cpu().numpy(), [u.cpu().numpy() for u in Us])
    rel_ref = O.rel_error(p.A, ref.G, ref.U)
    ang = max(float(O.principal_angles(u.cpu().numpy(), r).max()) for u, r in zip(Us, ref.U))
    sec, n = _oracle_time(lambda: O.st_hosvd_als(p.A, cfg.ranks, eta=cfg.eta, seed=1))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    _, fp64_peak = _alu_peaks(sms, clk.get("sm_mhz") or 2070.0)
    tf = fl / (pass_ms * 1e-3) / 1e12
    line = {"metric": "st-HOSVD-ALS time-to-tol (64^3 FP64)", "value": round(1e3 / ms, 2),
            "unit": "st-HOSVD/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": round(ms, 4), "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "st-HOSVD-ALS 64x64x64 FP64 rank (8,8,8) Gaussian core 1e-3 noise "
                                   "eta 1e-8", "sweeps": st["sweeps"], "l2": "L2 flushed between steps",
                       "rel_err": rel_own, "oracle_rel_err": rel_ref, "rel_err_gap": abs(rel_own - rel_ref),
                       "max_principal_angle": ang},
            "roofline": {"bound": "alu", "achieved": round(tf, 4), "peak": round(fp64_peak, 3),
                         "unit": "TFLOP/s", "frac": round(tf / fp64_peak, 4), "traffic": None,
                         "kernel": "tals::pass_kernel<double,...> (FP64 fused sweep, first mode, "
                                   "L2-resident when timed alone)",
                         "pass_ms": round(pass_ms, 5), "algorithmic_bytes": by, "algorithmic_flops": fl,
                         "peak_source": "nominal FP64 1.25 TFLOP/s at 2070 MHz, scaled to the SM clock"},
            "clocks": _clock_line(clk),
            "cpu_baseline": {"value": round(1.0 / sec, 2), "unit": "st-HOSVD/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": f"the full 64^3 decomposition, {n} runs"}}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_tucker(args):
    """Sec. 6.1.2's Tucker model at the paper's sizes: I x 100 x 100 x 100 FP32,
    I = 1000 .. 5000, truncation (I/100, 10, 10, 10), core U[5, 10], noise 1e-4,
    eta 1e-4; st- and t-HOSVD-ALS time-to-tol per size (the long first mode runs
    the two-pass sweep in t-HOSVD), errors against the input and the noiseless
    base. The line's value is st-HOSVD-ALS at I = 5000 (a 20 GB tensor)."""
    import numpy as np
    import torch
    import paper_2004_02583_gb300 as tals
    import workloads as W
    from oracle import tucker_oracle as O
    sizes = [int(x) for x in args.dims.split(",")] if args.dims else list(W.TUCKER_SIZES)
    peaks, _ = _peaks()
    clocks = Clocks(0)
    rows, roof, clk = [], None, {}
    for I in sizes:
        dims, ranks = (I, 100, 100, 100), (I // 100, 10, 10, 10)
        A = W.tucker_model_device(W.TUCKER_SEED + I, dims, ranks)
        G = torch.empty(ranks, device="cuda")
        Us = [torch.empty((d, r), device="cuda") for d, r in zip(dims, ranks)]
        res = {"I": I}
        for drv in ("st", "t"):
            ctx = tals.Context(A, ranks, eta=1e-4, seed=1)
            fn = (lambda: ctx.st_hosvd(G, Us)) if drv == "st" else (lambda: ctx.t_hosvd(G, Us))
            if I == sizes[-1] and drv == "st":
                clocks.start()
            ms, (_, _, st) = _time_gpu(fn, args.steps, args.warmup)
            if I == sizes[-1] and drv == "st":
                clk = clocks.stop()
                # the dominant kernel: the first mode's sweep pass over the whole tensor
                m0 = st["order"][0]
                pms, pby, _ = ctx.time_pass(mode=m0, iters=5)
                hbm = float(peaks.get("hbm_gbs", 6800.0))
                gbs = pby / (pms * 1e-3) / 1e9
                roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(gbs / hbm, 4), "traffic": None,
                        "kernel": f"tals::pass_kernel (fused FP32 sweep, mode {m0 + 1} of the "
                                  f"{I}x100x100x100 tensor, rank 10)",
                        "pass_ms": round(pms, 4), "algorithmic_bytes": pby,
                        "peak_source": f"HBM {hbm} GB/s (measured)"}
            b = tals.reconstruct(G, Us)
            base = W.tucker_model_device(W.TUCKER_SEED + I, dims, ranks, base_only=True)
            e_base = float(torch.linalg.vector_norm(b - base) / torch.linalg.vector_norm(base))
            del b, base
            res[drv] = {"ms": round(ms, 3), "rel_err": st["rel_err"], "err_vs_noiseless": e_base,
                        "sweeps": st["sweeps"]}
            ctx.close()
        rows.append(res)
        if I == sizes[0]:
            a_host = A.cpu().numpy().astype(np.float64)
        del A
        torch.cuda.empty_cache()
    # the oracle on the host on the smallest size, as it stands
    sec, n = _oracle_time(lambda: O.st_hosvd_als(a_host, (sizes[0] // 100, 10, 10, 10), eta=1e-4, seed=1))
    last = rows[-1]
    line = {"metric": "Tucker-model (Sec. 6.1.2) st-HOSVD-ALS time-to-tol",
            "value": round(1e3 / last["st"]["ms"], 3), "unit": "st-HOSVD/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": last["st"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"Tucker model {sizes[-1]}x100x100x100 FP32, ranks "
                                   f"({sizes[-1] // 100},10,10,10), core U[5,10], noise 1e-4, eta 1e-4",
                       "sizes": rows, "l2": "inputs (4-20 GB) larger than L2"},
            "roofline": roof, "clocks": _clock_line(clk),
            "cpu_baseline": {"value": round(1.0 / sec, 4), "unit": "st-HOSVD/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": f"FP64 NumPy oracle st-HOSVD-ALS on the {sizes[0]}x100x100x100 "
                                       f"tensor ({n} runs)"}}
    print(json.dumps(line), flush=True)


def run_rank500(args):
    """Sec. 6.4's dense test: a 5000 x 5000 x 50 FP32 Tucker tensor of multilinear
    rank (500, 500, 5) (the device-built Tucker model, noise 1e-2 of the base in
    norm), st-HOSVD-ALS (and one t-HOSVD-ALS run) at eta 1e-4 with the large-rank
    path for the two rank-500 modes; properties of the result (orthonormal
    factors, angles to the planted factors, error against the noiseless base).
    --dims I,J,K runs the same recipe at ranks (I/10, J/10, 5)."""
    import numpy as np
    import torch
    import paper_2004_02583_gb300 as tals
    import workloads as W
    from oracle import tucker_oracle as O
    dims = tuple(int(x) for x in args.dims.split(",")) if args.dims else W.RANK500_DIMS
    ranks = (dims[0] // 10, dims[1] // 10, 5) if args.dims else W.RANK500_RANKS
    delta = W.tucker_delta(dims, ranks, W.RANK500_NOISE)
    A, F = W.tucker_model_device(W.RANK500_SEED, dims, ranks, delta=delta, return_factors=True)
    peaks, _ = _peaks()
    clocks = Clocks(0)
    G = torch.empty(ranks, device="cuda")
    Us = [torch.empty((d, r), device="cuda") for d, r in zip(dims, ranks)]
    ctx = tals.Context(A, ranks, eta=1e-4, seed=1)
    clocks.start()
    ms, (_, _, st) = _time_gpu(lambda: ctx.st_hosvd(G, Us), args.steps, args.warmup)
    clk = clocks.stop()

    def props(G, Us):
        orth = max(float((u.double().T @ u.double() - torch.eye(u.shape[1], device="cuda",
                                                                  dtype=torch.float64)).abs().max()) for u in Us)
        sines = []
        for u, f in zip(Us, F):
            c = torch.linalg.svdvals((u.double().T @ f).cpu())
            sines.append(float(torch.sqrt(torch.clamp(1.0 - c.min() ** 2, min=0.0))))
        b = tals.reconstruct(G, Us)
        base = W.tucker_model_device(W.RANK500_SEED, dims, ranks, delta=delta, base_only=True)
        e_base = float(torch.linalg.vector_norm(b - base) / torch.linalg.vector_norm(base))
        e_in = float(torch.linalg.vector_norm(b - A) / torch.linalg.vector_norm(A))
        del b, base
        return {"max_orthonormality_defect": orth, "sin_max_angle_to_planted": sines,
                "rel_err_direct": e_in, "err_vs_noiseless": e_base}

    st_props = props(G, Us)
    # the rank-500 mode's products (mode 1 of the paper's numbering: the first
    # large-rank mode st-HOSVD reaches, on the tensor after the rank-5 mode)
    pm, pb, pf = ctx.time_sweep(mode=0, engine="cuda", iters=3)
    ctx.close()
    t_line = None
    if not args.no_compare:
        ctx = tals.Context(A, ranks, eta=1e-4, seed=1)
        tms, (_, _, tst) = _time_gpu(lambda: ctx.t_hosvd(G, Us), 1, 1)
        t_line = {"ms": round(tms, 3), "rel_err": tst["rel_err"], "sweeps": tst["sweeps"], **props(G, Us)}
        ctx.close()
    sm_mhz = clk.get("sm_mhz") or 2070.0
    alu, _ = _alu_peaks(152, sm_mhz)
    # mode 0 of the full tensor: the SGEMM pair of one sweep (2 I J R flops each)
    tf = [pf / 2.0 / (m * 1e-3) / 1e12 for m in pm]
    roof = {"bound": "alu", "achieved": round(tf[1], 2), "peak": round(alu, 2), "unit": "TFLOP/s",
            "frac": round(tf[1] / alu, 4), "traffic": None,
            "kernel": "cuBLAS SGEMM (pedantic FP32) of Y = B_(1) W over 2048-column ranges, mode 1 of the "
                      f"{'x'.join(map(str, dims))} tensor at rank {ranks[0]}",
            "w_product_ms": round(pm[0], 4), "y_product_ms": round(pm[1], 4),
            "w_product_tflops": round(tf[0], 2),
            "peak_source": f"FP32 FMA peak 152 SMs x 128 lanes x 2 flops x median SM clock {sm_mhz} MHz (derived)"}
    # the oracle as it stands, on the same recipe at 1/5 of each large mode
    sdims, sranks = (dims[0] // 5, dims[1] // 5, dims[2]), (ranks[0] // 5, ranks[1] // 5, ranks[2])
    a_small = W.tucker_model_device(W.RANK500_SEED, sdims, sranks,
                                    delta=W.tucker_delta(sdims, sranks, W.RANK500_NOISE)).cpu().numpy()
    sec, n = _oracle_time(lambda: O.st_hosvd_als(a_small.astype(np.float64), sranks, eta=1e-4, seed=1))

    def work(d, r):
        # sum over the st-HOSVD modes (ascending rank) of I_n J_n R_n of the current tensor
        d = list(d)
        tot = 0.0
        for m in sorted(range(3), key=lambda m: (r[m], m)):
            tot += float(np.prod(d)) * r[m]
            d[m] = r[m]
        return tot

    scale = work(dims, ranks) / work(sdims, sranks)
    line = {"metric": "Sec. 6.4 dense test st-HOSVD-ALS time-to-tol (ranks (500, 500, 5))",
            "value": round(1e3 / ms, 4), "unit": "st-HOSVD/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Tucker tensor {'x'.join(map(str, dims))} FP32, multilinear rank "
                                   f"{ranks}, core U[5,10], noise 1e-2 of the base, eta 1e-4",
                       "rel_err": st["rel_err"], "sweeps": st["sweeps"], "order": st["order"],
                       **st_props, "t_hosvd": t_line,
                       "l2": f"input ({A.numel() * 4 / 2**30:.1f} GiB) larger than L2"},
            "roofline": roof, "clocks": _clock_line(clk),
            "cpu_baseline": {"value": round(1.0 / (sec * scale), 6), "unit": "st-HOSVD/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": f"FP64 NumPy oracle st-HOSVD-ALS on the same recipe at "
                                       f"{'x'.join(map(str, sdims))}, ranks {sranks} ({n} runs of "
                                       f"{sec:.2f} s), scaled by {scale:.1f}, the ratio of the ALS "
                                       f"product work sum_n I_n J_n R_n"}}
    print(json.dumps(line), flush=True)


def _pass_rooflines(nctx, mctx, mode, sm_mhz, sms, peaks):
    pms, pby, pfl = nctx.time_pass(mode=mode, iters=10)
    tms, tby, tfl = mctx.time_pass(mode=mode, iters=10)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alu, _ = _alu_peaks(sms, sm_mhz)
    ptf = pfl / (pms * 1e-3) / 1e12
    pgb = pby / (pms * 1e-3) / 1e9
    tgb = tby / (tms * 1e-3) / 1e9
    roof = {"bound": "alu" if ptf / alu > pgb / hbm else "hbm",
            "achieved": round(ptf, 2) if ptf / alu > pgb / hbm else round(pgb, 1),
            "peak": round(alu, 2) if ptf / alu > pgb / hbm else hbm,
            "unit": "TFLOP/s" if ptf / alu > pgb / hbm else "GB/s",
            "frac": round(max(ptf / alu, pgb / hbm), 4), "traffic": None,
            "kernel": "tals::pass_kernel<float,...> (CUDA-core FP32 fused sweep, first mode)",
            "pass_ms": round(pms, 4), "hbm_gbs_achieved": round(pgb, 1),
            "alu_tflops_achieved": round(ptf, 2)}
    roof_tc = {"bound": "hbm", "achieved": round(tgb, 1), "peak": hbm, "unit": "GB/s",
               "frac": round(tgb / hbm, 4), "traffic": None,
               "kernel": "tals::tc_pass_kernel (tcgen05 BF16 sweep, first mode)", "pass_ms": round(tms, 4)}
    return roof, roof_tc


def run_c3(args):
    """128^4 FP32 rank (16,16,16,16), 0.8^k spectrum, 1e-3 noise: mixed vs plain."""
    import numpy as np
    import torch
    import paper_2004_02583_gb300 as tals
    import workloads as W
    from oracle import tucker_oracle as O
    cfg = W.CONFIGS["q128_f32"]
    p = W.make(cfg)
    A = torch.from_numpy(p.A).cuda()
    peaks, _ = _peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    G = torch.empty(cfg.ranks, device="cuda")
    Us = [torch.empty((d, r), device="cuda") for d, r in zip(cfg.dims, cfg.ranks)]
    res = {}
    clocks = Clocks(0)
    clocks.start()
    ctxs = {}
    precs = (args.precision,) if args.no_compare else ("mixed_bf16", "native")
    for prec in precs:
        ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision=prec,
                           use_graph=not args.no_graph)
        ms, (_, _, st) = _time_gpu(lambda: ctx.st_hosvd(G, Us), args.steps, args.warmup)
        res[prec] = (ms, st)
        ctxs[prec] = ctx
    clk = clocks.stop()
    if args.no_compare:
        print(json.dumps({"precision": args.precision, "ms_per_step": res[args.precision][0],
                          "sweeps": res[args.precision][1]["sweeps"]}))
        for c in ctxs.values():
            c.close()
        return
    roof, roof_tc = _pass_rooflines(ctxs["native"], ctxs["mixed_bf16"], res["native"][1]["order"][0],
                                    clk.get("sm_mhz") or 2070.0, sms, peaks)
    # oracle on a 128^3 x S slab of the same recipe, scaled to the full tensor
    S = 16
    q = W.planted(cfg.seed, cfg.dims[:3] + (S,), cfg.ranks, cfg.core, cfg.noise_rel, dtype=np.float32)
    a64 = q.A.astype(np.float64)
    sec, n = _oracle_time(lambda: O.st_hosvd_als(a64, cfg.ranks, eta=cfg.eta, seed=1), 10.0)
    mms, mst = res["mixed_bf16"]
    pms, pst = res["native"]
    line = {"metric": "st-HOSVD-ALS time-to-tol, mixed vs FP32 plain at equal error (128^4)",
            "value": round(1e3 / mms, 3), "unit": "st-HOSVD/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(mms, 4), "higher_is_better": True,
            "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": "st-HOSVD-ALS 128^4 FP32 rank (16,16,16,16) 0.8^k spectrum 1e-3 "
                                   "noise eta 1e-6", "l2": "inputs (1 GiB) larger than L2",
                       "mixed_ms": round(mms, 4), "fp32_plain_ms": round(pms, 4),
                       "speedup": round(pms / mms, 3), "mixed_rel_err": mst["rel_err"],
                       "fp32_plain_rel_err": pst["rel_err"],
                       "rel_err_gap": abs(mst["rel_err"] - pst["rel_err"]),
                       "sweeps": mst["sweeps"], "bulk_sweeps": mst["bulk_sweeps"],
                       "fp32_plain_sweeps": pst["sweeps"]},
            "roofline": roof, "roofline_tc": roof_tc, "clocks": _clock_line(clk),
            "cpu_baseline": {"value": (S / 128.0) / sec, "unit": "st-HOSVD/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": f"FP64 NumPy oracle on a 128^3 x {S} slab ({sec:.1f} s, {n} runs), "
                                       f"scaled by {S}/128"}}
    print(json.dumps(line), flush=True)
    for c in ctxs.values():
        c.close()


def run_c4(args):
    """4096 small FP32 tensors (modes ~ U{16..96}, ranks ~ U{4..16}): one batched
    graph-captured launch vs a per-tensor loop of the plain path."""
    import numpy as np
    import torch
    import paper_2004_02583_gb300 as tals
    import workloads as W
    from oracle import tucker_oracle as O
    count, eta = args.batch_count, 1e-6
    items = W.batched(W.SEED_BASE + 3, count)
    As = [torch.from_numpy(a).cuda() for a, _, _ in items]
    ranks = [r for _, _, r in items]
    clocks = Clocks(0)
    clocks.start()
    runner = tals.BatchedRunner(As, ranks, eta=eta, seed=1)
    ms, _ = _time_gpu(runner.run, args.steps, args.warmup)
    clk = clocks.stop()
    Gs, Us, sts = runner.Gs, runner.Us, runner.stats()
    # algorithmic bytes: every pass (initial guess + sweeps) reads the current tensor
    byt = 0
    for (a, dims, rk), st in zip(items, sts):
        cur = list(dims)
        for n in st["order"]:
            byt += (st["sweeps"][n] + 1) * int(np.prod(cur)) * 4
            cur[n] = rk[n]
    gbs = byt / (ms * 1e-3) / 1e9
    peaks, _ = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # per-tensor loop of the plain path on a subset, contexts made beforehand
    sub = min(256, count)
    ctxs = [tals.Context(As[t], ranks[t], eta=eta, seed=1) for t in range(sub)]
    loop_ms, _ = _time_gpu(lambda: [c.st_hosvd() for c in ctxs], 1, 1)
    loop_ms *= count / sub
    for c in ctxs:
        c.close()
    # parity on a few tensors against the oracle
    gaps = []
    for t in range(min(8, count)):
        a, dims, rk = items[t]
        ref = O.st_hosvd_als(a.astype(np.float64), rk, eta=eta, seed=1)
        own = O.rel_error(a.astype(np.float64), Gs[t].double().cpu().numpy(),
                          [u.double().cpu().numpy() for u in Us[t]])
        gaps.append(abs(own - O.rel_error(a.astype(np.float64), ref.G, ref.U)))
    osub = min(64, count)
    sec, n = _oracle_time(lambda: [O.st_hosvd_als(items[t][0].astype(np.float64), items[t][2], eta=eta,
                                                  seed=1) for t in range(osub)], 10.0)
    line = {"metric": f"batched st-HOSVD-ALS throughput ({count} uneven small tensors)",
            "value": round(count * 1e3 / ms, 1), "unit": "tensors/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(ms, 3), "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{count} x st-HOSVD-ALS FP32, I ~ U{{16..96}}, R ~ U{{4..16}}, 1e-2 noise, "
                                   "eta 1e-6, one persistent graph-captured launch",
                       "total_input_bytes": int(sum(a.nbytes for a, _, _ in items)),
                       "l2": "inputs (GBs) larger than L2",
                       "per_tensor_loop_ms": round(loop_ms, 2),
                       "per_tensor_loop_sample": f"{sub} tensors, scaled by {count}/{sub}",
                       "speedup_vs_loop": round(loop_ms / ms, 2),
                       "max_rel_err_gap_vs_oracle_8_tensors": max(gaps)},
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(gbs / hbm, 4), "traffic": None,
                         "kernel": "tals::batched_kernel (whole decomposition per CTA; algorithmic "
                                   "bytes = one read of the current tensor per pass)",
                         "algorithmic_bytes": byt},
            "clocks": _clock_line(clk),
            "cpu_baseline": {"value": round(osub / sec, 2), "unit": "tensors/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": f"FP64 NumPy oracle on the first {osub} tensors ({sec:.1f} s)"}}
    print(json.dumps(line), flush=True)


def run_c5(args):
    """1024x1024x512 FP32, rank (64,64,32): st-HOSVD-ALS forward, then the gradient
    of ||A - G x1 U1 x2 U2 x3 U3||^2 w.r.t. A and the factors through the
    projection / reconstruction kernels and their hand-written adjoints."""
    import numpy as np
    import torch
    import paper_2004_02583_gb300 as tals
    import workloads as W
    from oracle import tucker_oracle as O
    cfg = W.CONFIGS["d1024_f32"]
    if args.dims:   # profiling: the same recipe at other sizes
        p = W.planted(cfg.seed, tuple(int(x) for x in args.dims.split(",")), cfg.ranks, cfg.core,
                      cfg.noise_rel, dtype=np.float32)
    else:
        p = W.make(cfg)
    A = torch.from_numpy(p.A).cuda()
    if args.profile_pass:
        # only the Tucker mode products (two projections, two reconstructions), for an ncu capture
        rng = np.random.default_rng(0)
        Uq = [torch.from_numpy(np.linalg.qr(rng.standard_normal((d, r)))[0].astype(np.float32)).cuda()
              for d, r in zip(p.A.shape, cfg.ranks)]
        G = tals.project(A, Uq)
        tals.project(A, Uq)
        tals.reconstruct(G, Uq)
        tals.reconstruct(G, Uq)
        torch.cuda.synchronize()
        print(json.dumps({"profile_mode_products": list(p.A.shape)}))
        return
    peaks, _ = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    clocks = Clocks(0)
    clocks.start()
    ctx = tals.Context(A, cfg.ranks, eta=cfg.eta, seed=1, precision="native")
    fwd_ms, (G, Us, st) = _time_gpu(lambda: ctx.st_hosvd(), args.steps, args.warmup)
    Us = [u.detach().clone() for u in Us]

    def loss_and_grad():
        Ar = A.detach().requires_grad_(True)
        Ur = [u.detach().requires_grad_(True) for u in Us]
        # ||A - G x U||^2 with G = project(A, U): the fused loss kernel (the
        # reconstruction is never written), then the hand-written adjoints
        loss = tals.tucker_reconstruction_loss(Ar, tals.tucker_project(Ar, Ur), Ur)
        loss.backward()
        return Ar.grad, [u.grad for u in Ur]

    bwd_ms, _ = _time_gpu(loss_and_grad, max(3, args.steps // 2), args.warmup)
    # the reconstruction alone (writes the 2 GiB tensor): HBM-bound roofline
    Gd = G.detach().contiguous()
    rec_ms, _ = _time_gpu(lambda: tals.reconstruct(Gd, Us), args.steps, args.warmup)
    clk = clocks.stop()
    rec_bytes = A.numel() * 4 + Gd.numel() * 4 + sum(u.numel() * 4 for u in Us)
    gbs = rec_bytes / (rec_ms * 1e-3) / 1e9
    # algorithmic flops of the reconstruction in the library's mode order (the flop minimum over
    # all orders: each mode product costs 2 min(I_n, R_n) flops per element of its larger side)
    import itertools
    dims, rks = list(A.shape), list(cfg.ranks)

    def _order_flops(order):
        cur, fl = list(rks), 0
        for m in order:
            cur[m] = dims[m]
            fl += 2 * min(dims[m], rks[m]) * int(np.prod(cur))
        return fl
    rec_flops = min(_order_flops(o) for o in itertools.permutations(range(len(dims))))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    c5_mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = sms * 128 * 2 * c5_mhz * 1e6 / 1e12
    rec_tflops = rec_flops / (rec_ms * 1e-3) / 1e12
    # oracle: the loss gradient on a 1024 x 1024 x S slab, scaled
    S = 8
    a_s = p.A[:, :, :S].astype(np.float64)
    us_np = [u.double().cpu().numpy() for u in Us]
    us_s = [us_np[0], us_np[1], np.linalg.qr(us_np[2][:S])[0][:, :min(S, cfg.ranks[2])]]
    sec, n = _oracle_time(lambda: O.recon_loss_grad(a_s, us_s), 10.0)
    line = {"metric": "st-HOSVD-ALS forward + reconstruction-loss backward (1024x1024x512)",
            "value": round(1e3 / (fwd_ms + bwd_ms), 3), "unit": "forward+backward/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(fwd_ms + bwd_ms, 3),
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1024x1024x512 FP32 rank (64,64,32) 1/k spectrum 1e-2 noise eta 1e-6",
                       "forward_ms": round(fwd_ms, 3), "backward_ms": round(bwd_ms, 3),
                       "sweeps": st["sweeps"], "rel_err": st["rel_err"],
                       "l2": "inputs (2 GiB) larger than L2"},
            "roofline": {"bound": "alu", "achieved": round(rec_tflops, 2), "peak": round(alu_peak, 2),
                         "unit": "TFLOP/s", "frac": round(rec_tflops / alu_peak, 4),
                         # ncu DRAM bytes of the three mode products, from a capture of the
                         # 1024x1024x256 case, x2 for the full size
                         "traffic": 2 * (823040 + 8734720 + 73020000 + 134466304 + 1012872000),
                         "kernel": "reconstruct: three mg_pipe mode products (B = G x1 U1 x2 U2 x3 U3, "
                                   "2 GiB written; 64 flops per written element, above the SIMT ridge)",
                         "pass_ms": round(rec_ms, 3), "algorithmic_flops": rec_flops,
                         "algorithmic_bytes": rec_bytes, "hbm_gbs_achieved": round(gbs, 1),
                         "hbm_frac": round(gbs / hbm, 4),
                         "peak_source": f"FP32 FMA peak from {sms} SMs x 128 lanes x 2 flops x "
                                        f"{c5_mhz} MHz (derived); HBM {hbm} GB/s (measured)"},
            "clocks": _clock_line(clk),
            "cpu_baseline": {"value": round((S / 512.0) / sec, 4), "unit": "loss-gradients/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": f"FP64 NumPy oracle loss gradient on a 1024x1024x{S} slab "
                                       f"({sec:.1f} s, {n} runs), scaled by {S}/512"}}
    print(json.dumps(line), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
