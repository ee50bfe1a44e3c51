"""Benchmark: HBS build + preconditioned GMRES solve to 1e-10, in Mdof/s.

One step = ls_build (kernel spectrum, per-level compression, Algorithm 1) +
ls_solve (GMRES on the 10th-order FFT operator, right-preconditioned by the
HBS inverse, to relative residual 1e-10) + ls_free, on the workload
  precond_n256: 256 x 256 grid (N = 65,536) on the unit square, kappa = 60,
  b = 20 seeded Gaussians (seed 0) with a smooth cutoff, HBS eps = 1e-4 with
  4th-order corrections, matvec with 10th-order corrections, u_inc = e^{i kappa x1}.
value = N / (time per step) in Mdof/s for the mixed path (FP32 HBS, FP64 FFT
matvec and GMRES); the FP64 path is reported beside it.  Inputs (b, f) are
resident in device memory before the timed region; L2 is flushed (a 512 MB
write) between timed steps, outside the timed events.

--impl reference runs the CPU oracle (HBS + GMRES in numpy/scipy) on the same
workload on the host cores.
Multi-GPU: one process per GPU, each solving its own copy (replicas; the
path has no data exchange), value = all ranks' dofs / max-over-ranks time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HBS build+GMRES solve to 1e-10 (Mdof/s), mixed vs FP64 on GB300, % roofline"
WORKLOAD = "precond_n256"
WORKLOAD_TEXT = ("256x256 grid (N=65,536), kappa=60, b = 20 seeded Gaussians (seed 0) x smooth cutoff, "
                 "HBS eps=1e-4 order-4 corrections, FFT matvec order 10, plane wave theta=0, GMRES to 1e-10")
# Roofline denominators.  FP64 ALU: 1.25 TFLOP/s dense FP64 of a GB300 (nominal).
# FP32 SIMT: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s (unit
# counts and maximum clock).  TF32 tensor: half the bf16 dense rate.
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fp64_tflops": 1.25, "fp32_tflops": 80.5}


def max_over_ranks(values, world, device=None):
    """Per-rank times (s) reduced to their maximum over all ranks (every rank gets
    the result; an all-reduce on the default process group); unchanged at world 1."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput in millions of units per second: every rank (a replica)
    processed units_per_rank within `seconds`, the max over ranks."""
    return world * units_per_rank / seconds / 1e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return {"hbm_gbs": float(d.get("hbm_gbs", FALLBACK["hbm_gbs"])),
                    "bf16_tflops": float(d.get("bf16_tflops", FALLBACK["bf16_tflops"])),
                    "fp64_tflops": FALLBACK["fp64_tflops"], "fp32_tflops": FALLBACK["fp32_tflops"],
                    "source": "measured"}
        except Exception:
            pass
    return dict(FALLBACK, source="fallback")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_inputs():
    from paper_2007_12718_gb300 import inputs
    n, kappa = 256, 60.0
    return n, kappa, inputs.gaussian_family(n, 0)


# ----------------------------------------------------------------- reference
def oracle_step(n, kappa, b):
    from oracle import gmres, hbs, nystrom
    h = 1.0 / n
    comp = hbs.Compression(kappa, h, hbs.Tree(n, n, 8), 4, 1e-4, 2)
    inv = hbs.Inverse(comp, b)
    spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, 10)
    f = nystrom.rhs(kappa, b, n, n, h)
    s, k, hist = gmres.gmres(lambda v: nystrom.matvec_fft(spec, kappa, b, v), f, apply_M=inv.apply, tol=1e-10)
    return k


def cpu_baseline(n, kappa, b, reps=1):
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle_step(n, kappa, b)
    dt = (time.perf_counter() - t0) / reps
    return {"value": n * n / dt / 1e6, "unit": "Mdof/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} full build+solve of the same workload with the numpy/scipy oracle "
                      f"(BLAS/FFT threads: all {os.cpu_count()} cores), {dt:.2f} s each"}


def run_reference(args, rank):
    if rank != 0:
        return
    n, kappa, b = workload_inputs()
    for _ in range(args.warmup):
        oracle_step(n, kappa, b)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(n, kappa, b)
    dt = (time.perf_counter() - t0) / args.steps
    v = n * n / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mdof/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_TEXT},
            "cpu_baseline": {"value": v, "unit": "Mdof/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} full build+solve steps on the host cores"},
            "e2e": {"value": v, "unit": "Mdof/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- adjoint leg
ADJ_TEXT = ("512x512 grid, kappa=300, b = seed-0 Gaussian family, 32 plane waves theta_j = 2 pi j/32, "
            "256 receivers on the circle r=1.5 about (0.5,0.5), data = receiver field of the seed-1 potential; "
            "one step = ls_build + ls_set_receivers + ls_misfit_gradient (32 forward + 32 adjoint GMRES solves "
            "to 1e-10, receiver fields, gradient) + ls_free")


def adjoint_leg(ls, torch, dev, precision):
    """The differentiation workload: J(b) and dJ/db through the C ABI, timed with
    CUDA events on the current stream after one warm-up step (inputs resident)."""
    from paper_2007_12718_gb300 import inputs
    n, kappa, ndir, nrec = 512, 300.0, 32, 256
    h = 1.0 / n
    thetas = inputs.plane_wave_angles(ndir)
    rec = inputs.receivers_circle(nrec)
    b0 = torch.from_numpy(inputs.gaussian_family(n, 0)).to(dev)
    b1 = torch.from_numpy(inputs.gaussian_family(n, 1)).to(dev)
    H = ls.ls_build(n, h, kappa, b1, 1e-4, precision=precision)
    f = torch.zeros(ndir, n, n, dtype=torch.complex128, device=dev)
    ls.ls_rhs_plane_wave(H, thetas, f)
    sig = torch.zeros_like(f)
    ls.ls_solve(H, f, sig)
    ls.ls_set_receivers(H, rec)
    data = torch.zeros(ndir, nrec, dtype=torch.complex128, device=dev)
    ls.ls_receiver_field(H, sig, data)
    ls.ls_free(H)
    del f, sig
    grad = torch.zeros(n, n, dtype=torch.float64, device=dev)

    def step():
        Hs = ls.ls_build(n, h, kappa, b0, 1e-4, precision=precision)
        ls.ls_set_receivers(Hs, rec)
        out = ls.ls_misfit_gradient(Hs, thetas, data, grad)
        ls.ls_free(Hs)
        return out

    step()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    J, infos = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    fw = [i["iterations"] for i in infos[:ndir]]
    ad = [i["iterations"] for i in infos[ndir:]]
    return {"workload": "differentiation_n512", "description": ADJ_TEXT, "ms_per_gradient": ms,
            "value": ndir * n * n / (ms * 1e-3) / 1e6, "unit": "Mdof/s (directions x dofs, forward + adjoint)",
            "J": J, "gmres_iterations_forward_mean": float(np.mean(fw)),
            "gmres_iterations_adjoint_mean": float(np.mean(ad)),
            "converged": bool(all(i["converged"] for i in infos))}


# ----------------------------------------------------------------------- ours
def run_ours(args, rank, world):
    import torch

    import paper_2007_12718_gb300 as ls

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n, kappa, b = workload_inputs()
    N = n * n
    h = 1.0 / n
    stream = torch.cuda.current_stream()
    b_dev = torch.from_numpy(b).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # f = -kappa^2 b u_inc computed once on the device (input preparation, untimed)
    H0 = ls.ls_build(n, h, kappa, b_dev, 1e-4, precision=ls.LS_FP32)
    f_dev = torch.zeros(n, n, dtype=torch.complex128, device=dev)
    ls.ls_rhs_plane_wave(H0, [0.0], f_dev)
    ls.ls_free(H0)
    sig = torch.zeros(n, n, dtype=torch.complex128, device=dev)

    PREC = {"fp32": ls.LS_FP32, "tf32": ls.LS_TF32, "tf32x3": ls.LS_TF32X3}[args.precision]

    def step(precision):
        H = ls.ls_build(n, h, kappa, b_dev, 1e-4, precision=precision, top_uncompressed=args.top_uncompressed)
        info = ls.ls_solve(H, f_dev, sig)[0]
        ls.ls_free(H)
        return info

    def timed(precision, steps, profile=False):
        total = 0.0
        info = None
        if profile:
            ls.ls_profile_reset()
            ls.ls_profile_enable(True)
        launches0 = ls.ls_kernel_launches()
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step(precision)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        launches = ls.ls_kernel_launches() - launches0
        prof = None
        if profile:
            prof = ls.ls_profile_get()
            ls.ls_profile_enable(False)
        return total, info, launches, prof

    for _ in range(args.warmup):
        step(PREC)
        if not args.mixed_only:
            step(ls.LS_FP64)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t_mixed, info_mixed, launches, prof = timed(PREC, args.steps, profile=True)
    if world > 1:
        torch.distributed.barrier()
    steps64 = max(1, min(args.steps, 3))
    if args.mixed_only:
        t_fp64, info_fp64 = float("nan"), {"iterations": None, "resid_true": None}
    else:
        t_fp64, info_fp64, _, _ = timed(ls.LS_FP64, steps64, profile=True)

    # end to end through the public API with host buffers (b, f in pinned memory; sigma back)
    b_host = torch.from_numpy(b).pin_memory()
    f_host = f_dev.cpu().pin_memory()
    s_host = torch.zeros(n, n, dtype=torch.complex128).pin_memory()
    t_e2e = 0.0
    for _ in range(0 if args.mixed_only else args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = ls.ls_build(n, h, kappa, b_host, 1e-4, precision=PREC, top_uncompressed=args.top_uncompressed)
        ls.ls_solve(H, f_host, s_host)
        ls.ls_free(H)
        torch.cuda.synchronize()
        t_e2e += time.perf_counter() - t0

    t_mixed, t_fp64, t_e2e = max_over_ranks([t_mixed, t_fp64, t_e2e], world, dev)
    if rank != 0:
        return
    value = job_rate(world, N * args.steps, t_mixed)
    value64 = job_rate(world, N * steps64, t_fp64)
    e2e = job_rate(world, N * args.steps, t_e2e) if t_e2e > 0 else None

    # roofline of every timed kernel family; the one with the largest device time is the headline
    pk = peaks()
    tensor = args.precision in ("tf32", "tf32x3")

    def roof_of(name, p):
        avg_ms = p["total_ms"] / p["launches"]
        if name.startswith("matvec") or name == "spectrum_setup":
            bound, peak, unit, work = "alu", pk["fp64_tflops"], "TFLOP/s (FP64)", p["flops"]
            src = "nominal FP64 rate"
        elif name in ("hbs_apply", "gmres_orth"):
            bound, peak, unit, work = "hbm", pk["hbm_gbs"], "GB/s", p["bytes"]
            src = pk["source"]
        elif name == "merge_gemm" and tensor:
            bound, peak, unit, work = "tensor", pk["bf16_tflops"] / 2, "TFLOP/s (TF32)", p["flops"]
            src = pk["source"] + " bf16 x 1/2 (nominal tf32:bf16 ratio)"
        else:
            bound, peak, unit, work = "alu", pk["fp32_tflops"], "TFLOP/s (FP32 SIMT)", p["flops"]
            src = "unit counts x max clock"
        scale = 1e9 if unit == "GB/s" else 1e12
        achieved = work / p["launches"] / (avg_ms * 1e-3) / scale
        return {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None, "peak_source": src, "avg_launch_ms": avg_ms,
                "launches": p["launches"]}

    kernels = {k: roof_of(k, v) for k, v in prof.items() if v["launches"] > 0}
    single = {k: v for k, v in prof.items() if v["launches"] > 0 and k not in ("hbs_apply", "gmres_orth")}
    top = max(single.items(), key=lambda kv: kv[1]["total_ms"])[0]
    roof = kernels[top]
    breakdown = {k: round(v["total_ms"] / args.steps, 4) for k, v in prof.items() if v["launches"]}

    adj = adjoint_leg(ls, torch, dev, PREC) if not args.no_adjoint else None
    cpu = cpu_baseline(n, kappa, b) if not args.no_cpu_baseline else None
    line = {"metric": METRIC, "value": value, "unit": "Mdof/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_mixed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 HBS + c128 FFT/GMRES", "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_TEXT, "l2": "flushed between steps",
                       "top_levels_uncompressed": args.top_uncompressed,
                       "nrhs": 1, "precision": f"mixed ({args.precision} HBS merges, FP32 HBS storage, "
                                                        "FP64 matvec + GMRES)"},
            "fp64": {"value": value64, "unit": "Mdof/s", "ms_per_step": t_fp64 / steps64 * 1e3,
                     "iterations": info_fp64["iterations"], "resid_true": info_fp64["resid_true"]},
            "iterations": info_mixed["iterations"], "resid_true": info_mixed["resid_true"],
            "roofline": roof, "breakdown_ms_per_step": breakdown,
            "kernel_rooflines": {k: {"bound": v["bound"], "achieved": round(v["achieved"], 3), "unit": v["unit"],
                                     "frac": round(v["frac"], 4)} for k, v in kernels.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "Mdof/s", "h2d_bytes_per_step": N * 8 + N * 16,
                    "d2h_bytes_per_step": N * 16},
            "gpu_launches": launches, "clocks": clk.summary(), "adjoint": adj}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the differentiation workload (512x512 misfit gradient) reported under 'adjoint'")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32", "tf32x3"],
                    help="engine of the mixed path's merge GEMMs (FP32 storage in all three)")
    ap.add_argument("--top-uncompressed", type=int, default=1,
                    help="tree levels kept uncompressed at the top (U = I); 0 = every level compressed")
    ap.add_argument("--mixed-only", action="store_true",
                    help="time only the mixed path (no FP64 or end-to-end legs); for profiler runs")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
