"""Benchmark: HBS build + preconditioned GMRES solve to 1e-10, in Mdof/s, mixed vs FP64.

One step = ls_build (corrected-quadrature weights, kernel spectrum, per-level
compression, Algorithm 1) + ls_solve (GMRES on the 10th-order FFT operator,
right-preconditioned by the HBS inverse, to relative residual 1e-10) + ls_free.

Headline workload precond_n2048: 2048 x 2048 grid (N = 4,194,304) on the unit
square, kappa = 400 pi (200 wavelengths across, 10.24 points per wavelength),
b = 20 seeded Gaussians (seed 0) with a smooth cutoff, HBS eps = 1e-4 with
4th-order corrections, matvec with 10th-order corrections, u_inc = e^{i kappa x1}.
value = N / (device time per step) in Mdof/s for the mixed path (FP32 HBS with
tf32x3 tensor-core merge GEMMs, FP64 FFT matvec and GMRES), timed with CUDA
events with no per-kernel profiling; the plain FP64 path is measured on the same
workload beside it (`fp64`).  A separate profiled pass gives the per-phase and
end-to-end rooflines.  Inputs (b, f) are resident in device memory before the
timed region; L2 is flushed (a 512 MB write) between timed steps, outside the
timed events (the factors, ~30 GB, are far larger than L2 anyway).
Secondary legs: precond_n256 (256^2, kappa 60), direct_n32 (HBS direct solve at
eps 1e-10), differentiation_n512 (misfit gradient by the adjoint method).

--impl reference runs the CPU oracle (HBS + GMRES in numpy/scipy) on bounded
samples of the workload on the host cores (see cpu_sample_step).
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
WORKLOAD = "precond_n2048"
WORKLOAD_TEXT = ("2048x2048 grid (N=4,194,304), kappa=400 pi (200 wavelengths, 10.24 points per wavelength), "
                 "b = 20 seeded Gaussians (seed 0) x smooth cutoff, HBS eps=1e-4 order-4 corrections, FFT matvec "
                 "order 10, plane wave theta=0, GMRES to 1e-10")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


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


def file_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                    "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                    "source": "of measured (MEASURED_PEAKS.json)"}
        except Exception:
            pass
    return dict(FALLBACK, bf16_tflops_sustained=1700.0, source="of fallback")


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


def workload(name):
    from paper_2007_12718_gb300 import inputs
    w = inputs.WORKLOADS[name]
    return w["n"], w["kappa"], w["b"](w["n"]), w


# ----------------------------------------------------------------- reference
CPU_SAMPLE = "precond_n256_10ppw"
CPU_SAMPLE_TEXT = ("one full HBS build + preconditioned GMRES solve by the numpy/scipy oracle on the 256x256 member "
                   "of the same workload family at the same kappa h (kappa = 50 pi, 10.24 points per wavelength, "
                   "seed-0 potential, eps 1e-4); Mdof/s = 256^2 / its time.  The oracle's cost grows like N^1.5, so "
                   "this sample overstates its rate at 2048^2")


def cpu_sample_step():
    """The oracle's complete method (Algorithms 1-2 with scipy CPQR, FFT matvec,
    GMRES) on the bounded sample; returns (seconds, iterations)."""
    from oracle import gmres, hbs, nystrom
    n, kappa, b, w = workload(CPU_SAMPLE)
    h = 1.0 / n
    t0 = time.perf_counter()
    comp = hbs.Compression(kappa, h, hbs.Tree(n, n, w["leaf"]), w["order_precond"], w["eps"], 2)
    inv = hbs.Inverse(comp, b)
    spec = nystrom.conv_kernel_spectrum(kappa, h, n, n, w["order_matvec"])
    f = nystrom.rhs(kappa, b, n, n, h)
    s, k, hist = gmres.gmres(lambda v: nystrom.matvec_fft(spec, kappa, b, v), f, apply_M=inv.apply, tol=1e-10)
    return time.perf_counter() - t0, k


def cpu_baseline():
    dt, k = cpu_sample_step()
    n = workload(CPU_SAMPLE)[0]
    return {"value": n * n / dt / 1e6, "unit": "Mdof/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": CPU_SAMPLE_TEXT + f"; {dt:.2f} s, {k} GMRES iterations, BLAS/FFT threads: all "
                                        f"{os.cpu_count()} cores"}


def run_reference(args, rank):
    if rank != 0:
        return
    n = workload(CPU_SAMPLE)[0]
    for _ in range(args.warmup):
        cpu_sample_step()
    t = 0.0
    for _ in range(args.steps):
        dt, k = cpu_sample_step()
        t += dt
    dt = t / args.steps
    v = n * n / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mdof/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_TEXT, "sample": CPU_SAMPLE_TEXT},
            "cpu_baseline": {"value": v, "unit": "Mdof/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": CPU_SAMPLE_TEXT + f"; {args.steps} timed samples after {args.warmup}"},
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


# ------------------------------------------------------------ multi-RHS leg
MRHS_TEXT = ("512x512 grid, kappa=300, b = seed-0 Gaussian family, 256 plane waves theta_j = 2 pi j/256 as one "
             "block; one step = ls_build + ls_rhs_plane_wave + ls_solve (block GMRES to 1e-10 for every direction, "
             "block apply: each factor read once per iteration for all 256) + ls_free")


def multirhs_leg(ls, torch, dev, precision, flush, pk, tensor):
    """Many incident fields on one factorisation, timed with CUDA events after one
    warm-up step (inputs resident); the same with one right-hand side at a time for
    comparison, and a profiled step for the phase rooflines."""
    from paper_2007_12718_gb300 import inputs
    w = inputs.WORKLOADS["multirhs_n512"]
    n, kappa, nr = w["n"], w["kappa"], w["nrhs"]
    h = 1.0 / n
    th = inputs.plane_wave_angles(nr)
    b = torch.from_numpy(w["b"](n)).to(dev)
    F = torch.zeros(nr, n, n, dtype=torch.complex128, device=dev)
    sig = torch.zeros_like(F)
    stream = torch.cuda.current_stream()

    def step(blk):
        H = ls.ls_build(n, h, kappa, b, w["eps"], precision=precision, rhs_block=blk)
        ls.ls_rhs_plane_wave(H, th, F)
        infos = ls.ls_solve(H, F, sig)
        ls.ls_free(H)
        return infos

    def timed(blk, profile=False):
        if profile:
            ls.ls_profile_reset()
            ls.ls_profile_enable(True)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = step(blk)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = None
        if profile:
            prof = ls.ls_profile_get()
            ls.ls_profile_enable(False)
        return e0.elapsed_time(e1) * 1e-3, infos, prof

    step(0)
    t, infos, _ = timed(0)
    t1, infos1, _ = timed(1)
    _, _, prof = timed(0, profile=True)
    fams, phases, _ = rooflines(prof, pk, tensor, t, 1)
    its = [i["iterations"] for i in infos]
    return {"workload": "multirhs_n512", "description": MRHS_TEXT, "nrhs": nr, "ms_per_step": t * 1e3,
            "value": nr * n * n / t / 1e6, "unit": "Mdof/s (directions x dofs, build + solve)",
            "one_at_a_time": {"ms_per_step": t1 * 1e3, "value": nr * n * n / t1 / 1e6},
            "iterations_min": min(its), "iterations_max": max(its),
            "resid_true_max": max(i["resid_true"] for i in infos),
            "converged": bool(all(i["converged"] for i in infos)),
            "phase_rooflines": phases,
            "kernel_rooflines": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                                 for k, v in fams.items()}}


# --------------------------------------------------------- multi-problem leg
MPROB_TEXT = ("32 independent problems, sides drawn from {64, 96, 128, 192} (default_rng(7)), kappa = 2 pi n/10 "
              "(10 points per wavelength), b = Gaussian family seeds 100..131, theta = 0, leaf side 8 or 12; one "
              "step = per side one ls_build_many (a forest of that side's problems: one compression, batched "
              "merges) + ls_rhs_plane_wave + ls_solve (block GMRES, one right-hand side per problem) + ls_free")


def multiproblem_leg(ls, torch, dev, precision, flush):
    """Many independent problems of uneven sizes: grouped by side into forests,
    timed with CUDA events after one warm-up step; the same problems one handle
    each for comparison."""
    from paper_2007_12718_gb300 import inputs
    probs = inputs.multiproblem_set()
    groups = {}
    for p in probs:
        groups.setdefault(p["n"], []).append(p)
    data = {}
    for n, grp in groups.items():
        bs = torch.from_numpy(np.stack([inputs.gaussian_family(n, p["b_seed"]) for p in grp])).to(dev)
        data[n] = (grp, bs, torch.zeros(len(grp), n, n, dtype=torch.complex128, device=dev),
                   torch.zeros(len(grp), n, n, dtype=torch.complex128, device=dev))
    stream = torch.cuda.current_stream()

    def step(forest):
        infos = []
        for n, (grp, bs, F, sig) in data.items():
            kw = dict(leaf_side=grp[0]["leaf"], precision=precision)
            if forest:
                H = ls.ls_build(n, 1.0 / n, grp[0]["kappa"], bs, 1e-4, **kw)
                ls.ls_rhs_plane_wave(H, [0.0], F)
                infos += ls.ls_solve(H, F, sig)
                ls.ls_free(H)
            else:
                for g in range(len(grp)):
                    H = ls.ls_build(n, 1.0 / n, grp[0]["kappa"], bs[g], 1e-4, **kw)
                    ls.ls_rhs_plane_wave(H, [0.0], F[g])
                    infos += ls.ls_solve(H, F[g], sig[g])
                    ls.ls_free(H)
        return infos

    def timed(forest):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = step(forest)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3, infos

    step(True)
    step(False)
    t, infos = timed(True)
    t1, _ = timed(False)
    dofs = sum(p["n"] ** 2 for p in probs)
    return {"workload": "multiproblem_32", "description": MPROB_TEXT, "problems": len(probs),
            "sides": {str(n): len(g) for n, g in sorted(groups.items())}, "dofs": dofs,
            "ms_per_step": t * 1e3, "value": dofs / t / 1e6, "unit": "Mdof/s (all problems, build + solve)",
            "one_handle_per_problem": {"ms_per_step": t1 * 1e3, "value": dofs / t1 / 1e6},
            "converged": bool(all(i["converged"] for i in infos)),
            "resid_true_max": max(i["resid_true"] for i in infos),
            "iterations_max": max(i["iterations"] for i in infos)}


# ----------------------------------------------------------------------- ours
class Leg:
    """One workload on the device: inputs resident, steps of build + solve + free."""

    def __init__(self, ls, torch, dev, name, precision, **build_kw):
        self.ls, self.torch, self.dev = ls, torch, dev
        self.n, self.kappa, b, self.w = workload(name)
        self.N = self.n * self.n
        self.h = 1.0 / self.n
        self.precision = precision
        self.kw = dict(order_precond=self.w["order_precond"], order_matvec=self.w["order_matvec"],
                       leaf_side=self.w["leaf"], **build_kw)
        self.b_np = b
        self.b = torch.from_numpy(b).to(dev)
        self.f = None
        self.sig = torch.zeros(self.n, self.n, dtype=torch.complex128, device=dev)

    def step(self, precision=None):
        ls = self.ls
        H = ls.ls_build(self.n, self.h, self.kappa, self.b, self.w["eps"],
                        precision=self.precision if precision is None else precision, **self.kw)
        if self.f is None:  # f = -kappa^2 b u_inc on the device, once (input preparation, untimed warm-up)
            self.f = self.torch.zeros(self.n, self.n, dtype=self.torch.complex128, device=self.dev)
            ls.ls_rhs_plane_wave(H, [0.0], self.f)
        info = ls.ls_solve(H, self.f, self.sig)[0]
        binfo = H.info()
        ls.ls_free(H)
        return info, binfo

    def timed(self, steps, flush, stream, precision=None, profile=False):
        ls, torch = self.ls, self.torch
        total, info, binfo = 0.0, None, None
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
            info, binfo = self.step(precision)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        launches = ls.ls_kernel_launches() - launches0
        prof = None
        if profile:
            prof = ls.ls_profile_get()
            ls.ls_profile_enable(False)
        return total, info, binfo, launches, prof

    def e2e(self, steps, flush):
        """Through the C ABI with host buffers: b and f from pinned host memory,
        sigma back to pinned host memory, copies inside the timed region."""
        ls, torch = self.ls, self.torch
        b_host = torch.from_numpy(self.b_np).pin_memory()
        f_host = self.f.cpu().pin_memory()
        s_host = torch.zeros(self.n, self.n, dtype=torch.complex128).pin_memory()
        t = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H = ls.ls_build(self.n, self.h, self.kappa, b_host, self.w["eps"], precision=self.precision, **self.kw)
            ls.ls_solve(H, f_host, s_host)
            ls.ls_free(H)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
        return t, {"h2d_bytes_per_step": self.N * 8 + self.N * 16, "d2h_bytes_per_step": self.N * 16}


# DRAM traffic of a kernel family per build + solve step, from one ncu capture of the same command
# (dram__bytes_read.sum + dram__bytes_write.sum); keyed by (workload, precision, family).
MEASURED_TRAFFIC = {
    ("precond_n2048", "tf32x3", "merge_gemm"): {
        "bytes": 99.18e9,
        "note": "bytes per build + solve step of the 271 tcgen05 GEMM launches (ncu, one-pass metrics at full "
                "size; profiles/tc_gemm_traffic_precond_n2048.md); ~250 algorithmic flops per DRAM byte"},
    ("precond_n2048", "tf32x3", "cpqr_id"): {
        "bytes": 148.96e9,
        "note": "bytes per build + solve step of the compression's blocked row IDs and interpolation matrices "
                "(ncu, one-pass metrics at full size, split by stream; profiles/blocked_id_traffic_precond_n2048.md): "
                "13.5x the algorithmic bytes, each block of 32 pivots passing over the trailing candidates"},
}

# phases of the method and the kernel families of each
PHASES = {
    "compress": ["cpqr_id"],
    "merges": ["leaf_build", "merge_gemm", "merge_inverse"],
    "apply": ["hbs_apply", "hbs_apply_block"],
    "matvec": ["matvec_rows_fwd", "matvec_cols", "matvec_rows_inv", "spectrum_setup"],
    "gmres": ["gmres_orth", "gmres_block"],
}


def family_peak(name, pk, tensor):
    """(bound, peak, unit, source) of a kernel family's roofline."""
    if name.startswith("matvec") or name == "spectrum_setup":
        return "alu", pk["fp64_tflops"], "TFLOP/s (FP64)", "of measured (ls_measure_peak FP64 FMA loop)"
    if name in ("hbs_apply", "gmres_orth", "gmres_block"):
        return "hbm", pk["hbm_gbs"], "GB/s", pk["source"]
    if name in ("merge_gemm", "hbs_apply_block") and tensor:
        return ("tensor", pk["bf16_tflops"] / 2, "TFLOP/s (TF32 dense)",
                pk["source"] + " bf16 x 1/2 (nominal tf32:bf16 ratio)")
    return "alu", pk["fp32_tflops"], "TFLOP/s (FP32)", "of measured (ls_measure_peak packed FP32 FMA loop)"


def rooflines(prof, pk, tensor, t_total, steps):
    fams = {}
    for k, v in prof.items():
        if v["launches"] <= 0 or v["total_ms"] <= 0:
            continue
        bound, peak, unit, src = family_peak(k, pk, tensor)
        work = v["bytes"] if unit == "GB/s" else v["flops"]
        scale = 1e9 if unit == "GB/s" else 1e12
        achieved = work / (v["total_ms"] * 1e-3) / scale
        fams[k] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                   "peak_source": src, "ms_per_step": v["total_ms"] / steps, "launches": v["launches"],
                   "work_per_step": work / steps, "min_s_per_step": work / steps / (peak * scale)}
    phases = {}
    ideal = 0.0
    for ph, names in PHASES.items():
        sel = [fams[n] for n in names if n in fams]
        if not sel:
            continue
        ms = sum(f["ms_per_step"] for f in sel)
        mins = sum(f["min_s_per_step"] for f in sel)
        ideal += mins
        phases[ph] = {"ms_per_step": ms, "min_ms_at_peak": mins * 1e3, "frac": mins / (ms * 1e-3)}
    e2e = {"t_step_s": t_total, "min_s_at_peaks": ideal, "frac": ideal / t_total,
           "note": "sum over phases of (algorithmic work / peak), over the measured step time"}
    return fams, phases, e2e


def measured_peaks(ls):
    pk = file_peaks()
    pk["fp64_tflops"] = ls.ls_measure_peak(0)
    pk["fp32_scalar_tflops"] = ls.ls_measure_peak(1)
    pk["fp32_tflops"] = max(pk["fp32_scalar_tflops"], ls.ls_measure_peak(2))
    return pk


def run_ours(args, rank, world):
    import torch

    import paper_2007_12718_gb300 as ls

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if args.precision == "fp64":
        raise SystemExit("--precision fp64 is for --sweep; the benchmark measures the FP64 path beside the mixed one")
    PREC = {"fp32": ls.LS_FP32, "tf32x3": ls.LS_TF32X3, "fp16split": ls.LS_FP16SPLIT}[args.precision]
    tensor = args.precision in ("tf32x3", "fp16split")
    pk = measured_peaks(ls)

    main = Leg(ls, torch, dev, args.workload, PREC, top_uncompressed=args.top_uncompressed)
    for _ in range(args.warmup):
        main.step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t_mixed, info_mixed, binfo, launches, _ = main.timed(args.steps, flush, stream)
    if world > 1:
        torch.distributed.barrier()
    sig_mixed = main.sig.clone()
    # profiled pass (per-launch events on): the phase breakdown and the rooflines
    t_prof, _, _, _, prof = main.timed(1, flush, stream, profile=True)
    # the plain FP64 path on the same workload
    t_fp64, info_fp64, fp64_steps = float("nan"), None, 0
    agree = None
    if args.fp64_steps > 0:
        for _ in range(args.fp64_warmup):
            main.step(ls.LS_FP64)
        t_fp64, info_fp64, _, _, _ = main.timed(args.fp64_steps, flush, stream, precision=ls.LS_FP64)
        fp64_steps = args.fp64_steps
        agree = float(torch.linalg.norm(main.sig - sig_mixed) / torch.linalg.norm(main.sig))
    # the FP16 split-product engine on the same workload (one warm-up, one timed step)
    f16 = None
    if args.fp16_steps > 0:
        main.step(ls.LS_FP16SPLIT)
        t16, info16, _, _, _ = main.timed(args.fp16_steps, flush, stream, precision=ls.LS_FP16SPLIT)
        f16 = {"value": main.N * args.fp16_steps / t16 / 1e6, "unit": "Mdof/s", "steps": args.fp16_steps,
               "ms_per_step": t16 / args.fp16_steps * 1e3, "iterations": info16["iterations"],
               "resid_true": info16["resid_true"],
               "sigma_rel_diff_vs_mixed": float(torch.linalg.norm(main.sig - sig_mixed) / torch.linalg.norm(sig_mixed)),
               "precision": "FP16 split products (kind::f16 hi/lo, power-of-two operand scales), FP32 HBS"}
    t_e2e, e2e_bytes = main.e2e(args.e2e_steps, flush) if args.e2e_steps > 0 else (0.0, None)

    t_mixed, t_fp64, t_e2e = max_over_ranks([t_mixed, t_fp64, t_e2e], world, dev)
    if rank != 0:
        return
    N = main.N
    value = job_rate(world, N * args.steps, t_mixed)
    value64 = job_rate(world, N * fp64_steps, t_fp64) if fp64_steps else None
    e2e = job_rate(world, N * args.e2e_steps, t_e2e) if t_e2e > 0 else None
    fams, phases, e2e_roof = rooflines(prof, pk, tensor, t_mixed / args.steps, 1)
    top = max((k for k in fams if k not in ("hbs_apply", "gmres_orth")), key=lambda k: fams[k]["ms_per_step"])
    f = fams[top]
    traffic = MEASURED_TRAFFIC.get((args.workload, args.precision, top))
    roof = {"bound": f["bound"], "kernel": top, "achieved": f["achieved"], "peak": f["peak"], "unit": f["unit"],
            "frac": f["frac"], "traffic": traffic["bytes"] if traffic else None, "peak_source": f["peak_source"],
            "note": "achieved = the family's algorithmic work over its device time in the profiled pass"}
    if traffic:
        roof["traffic_note"] = traffic["note"]

    secondary = {}
    if not args.no_secondary:
        for name, prec_list in (("precond_n256", [PREC, ls.LS_FP64]),):
            leg = Leg(ls, torch, dev, name, PREC, top_uncompressed=args.top_uncompressed)
            out = {}
            for pr in prec_list:
                for _ in range(2):
                    leg.step(pr)
                t, info, bi, _, _ = leg.timed(3, flush, stream, precision=pr)
                out["mixed" if pr == PREC else "fp64"] = {
                    "value": leg.N * 3 / t / 1e6, "unit": "Mdof/s", "ms_per_step": t / 3 * 1e3,
                    "iterations": info["iterations"], "resid_true": info["resid_true"], "ranks": bi["ranks"]}
            secondary[name] = out
        leg = Leg(ls, torch, dev, "direct_n32", ls.LS_FP64)
        leg.step()
        t, info, bi, _, _ = leg.timed(3, flush, stream)
        secondary["direct_n32"] = {"value": leg.N * 3 / t / 1e6, "unit": "Mdof/s", "ms_per_step": t / 3 * 1e3,
                                   "precision": "FP64, eps 1e-10, order-10 corrections inside the HBS",
                                   "iterations": info["iterations"], "resid_true": info["resid_true"]}
    adj = adjoint_leg(ls, torch, dev, PREC) if not args.no_adjoint else None
    if adj:
        secondary["differentiation_n512"] = adj
    if not args.no_multirhs:
        secondary["multirhs_n512"] = multirhs_leg(ls, torch, dev, PREC, flush, pk, tensor)
    if not args.no_multiproblem:
        secondary["multiproblem_32"] = multiproblem_leg(ls, torch, dev, PREC, flush)
    cpu = cpu_baseline() if not args.no_cpu_baseline else None
    line = {"metric": METRIC, "value": value, "unit": "Mdof/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_mixed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 HBS + c128 FFT/GMRES", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOAD_TEXT if args.workload == WORKLOAD else
                       args.workload, "l2": "flushed between steps (inputs and factors also far larger than L2)",
                       "nrhs": 1, "precision": f"mixed ({args.precision} merge GEMMs, FP32 HBS, FP64 matvec + GMRES)",
                       "top_levels_uncompressed": args.top_uncompressed},
            "iterations": info_mixed["iterations"], "resid_true": info_mixed["resid_true"],
            "ranks": binfo["ranks"], "factor_GB": binfo["factor_bytes"] / 1e9,
            "fp64": {"value": value64, "unit": "Mdof/s", "steps": fp64_steps, "warmup": args.fp64_warmup,
                     "ms_per_step": t_fp64 / fp64_steps * 1e3 if fp64_steps else None,
                     "iterations": info_fp64["iterations"] if info_fp64 else None,
                     "resid_true": info_fp64["resid_true"] if info_fp64 else None,
                     "sigma_rel_diff_mixed_vs_fp64": agree},
            "fp16split": f16,
            "roofline": roof, "phase_rooflines": phases, "e2e_roofline": e2e_roof,
            "kernel_rooflines": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                                 for k, v in fams.items()},
            "profiled_step_ms": t_prof * 1e3,
            "peaks": pk,
            "cpu_baseline": cpu,
            "e2e": dict({"value": e2e, "unit": "Mdof/s", "steps": args.e2e_steps}, **(e2e_bytes or {})),
            "gpu_launches": launches, "clocks": clk.summary(), "secondary": secondary}
    print(json.dumps(line), flush=True)


# The paper's cavity table (Sec. 6.3, preconditioned solver, 10 points per
# wavelength): N, kappa, T_skel + T_build, T_gmres (s, 36-core workstation), iterations.
PAPER_CAVITY = {6400: (0.47, 0.20, 4), 25600: (1.64, 0.62, 5), 102400: (6.62, 2.49, 6), 409600: (34.97, 9.78, 6),
                1638400: (190.38, 56.13, 9), 6553600: (829.48, 330.91, 13), 26214400: (5126.25, 2698.53, 22)}


# The paper's lens table (Sec. 6.2 test problems, kappa = 300): N -> GMRES iterations.
PAPER_LENS = {102400: 51, 409600: 9, 1638400: 7, 6553600: 7, 26214400: 9}


# The paper's direct-solver tables (Sec. 6.1, Gaussian bump, kappa = 25): (eps, N) ->
# (T_skel + T_build, T_apply, residual); 36-core workstation.
PAPER_DIRECT = {
    (1e-3, 6400): (1.75, 0.05, 7.74e-05), (1e-3, 25600): (7.28, 0.12, 5.71e-05),
    (1e-3, 102400): (37.85, 0.48, 9.75e-05), (1e-3, 409600): (167.85, 2.00, 1.56e-04),
    (1e-6, 6400): (3.16, 0.07, 9.54e-09), (1e-6, 25600): (16.00, 0.19, 7.13e-08),
    (1e-6, 102400): (79.25, 0.76, 4.15e-08), (1e-6, 409600): (443.86, 6.58, 4.39e-08),
    (1e-9, 6400): (4.04, 0.07, 1.57e-12), (1e-9, 25600): (23.39, 0.24, 3.37e-12),
    (1e-9, 102400): (117.57, 1.04, 1.45e-11), (1e-9, 409600): (675.66, 6.82, 3.48e-09),
    (1e-12, 6400): (4.40, 0.07, 1.87e-15), (1e-12, 25600): (23.70, 0.22, 3.80e-15),
    (1e-12, 102400): (125.78, 1.00, 6.94e-15), (1e-12, 409600): (767.18, 5.98, 1.71e-14),
    (1e-3, 1638400): (845.19, 10.53, 5.77e-04), (1e-6, 1638400): (2791.95, 33.50, 3.14e-07),
    (1e-9, 1638400): (4162.88, 67.17, 2.99e-09), (1e-12, 1638400): (4778.64, 47.13, 5.07e-14),
}


def run_direct_sweep(args):
    """The direct solver of Sec. 6.1: b = 1.5 exp(-160 |x|^2), kappa = 25, 10th-order
    corrections inside the HBS and in the operator, 100-point leaves, eps = 1e-3 ... 1e-12,
    n = 80 2^j.  FP32 storage (tf32x3 merges) for eps = 1e-3, FP64 below.  Per size: build
    time, one apply, and the residual ||f - A M f|| / ||f|| of the direct solution M f
    (f = -kappa^2 b u_inc), CUDA events after one warm-up.  One JSON line."""
    import torch

    import paper_2007_12718_gb300 as ls
    from paper_2007_12718_gb300 import inputs

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    rows = []
    kappa = 25.0
    eps_list = [float(e) for e in args.sweep_eps.split(",")] if args.sweep_eps else [1e-3, 1e-6, 1e-9, 1e-12]
    for eps in eps_list:
        prec = ls.LS_TF32X3 if eps >= 1e-3 else ls.LS_FP64
        # n <= 640 by default; 1280 (the paper's largest, 1,638,400 unknowns) with --sweep-levels 5
        for j in range(args.sweep_first, min(args.sweep_levels, 5) if args.sweep_eps else min(args.sweep_levels, 4)):
            n = 80 << j
            h = 1.0 / n
            b = torch.from_numpy(inputs.gaussian_direct(n)).to(dev)
            f = torch.zeros(n, n, dtype=torch.complex128, device=dev)
            q = torch.zeros_like(f)
            y = torch.zeros_like(f)
            tb = ta = 0.0
            for it in range(2):
                torch.cuda.synchronize()
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
                H = ls.ls_build(n, h, kappa, b, eps, leaf_side=10, order_precond=10, order_matvec=10, precision=prec)
                e[1].record(stream)
                if it == 0:
                    ls.ls_rhs_plane_wave(H, [0.0], f)
                    ls.ls_apply(H, f, q)  # warm-up of the apply
                    torch.cuda.synchronize()
                    e[1].record(stream)
                ls.ls_apply(H, f, q)
                e[2].record(stream)
                torch.cuda.synchronize()
                if it == 1:
                    tb, ta = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
                    ls.ls_matvec(H, q, y)
                    res = float(torch.linalg.norm(f - y) / torch.linalg.norm(f))
                    bi = H.info()
                ls.ls_free(H)
            paper = PAPER_DIRECT.get((eps, n * n))
            rows.append({"eps": eps, "N": n * n, "precision": "tf32x3" if prec == ls.LS_TF32X3 else "fp64",
                         "t_build_s": tb, "t_apply_s": ta, "residual": res, "factor_GB": bi["factor_bytes"] / 1e9,
                         "ranks_top": bi["ranks"][1:4],
                         "paper": None if paper is None else {"t_skel_plus_build_s": paper[0], "t_apply_s": paper[1],
                                                              "residual": paper[2]}})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del b, f, q, y
            torch.cuda.empty_cache()
    print(json.dumps({"metric": METRIC, "sweep": "direct solver, Gaussian bump, kappa = 25 (Sec. 6.1)",
                      "rows": rows}), flush=True)


def run_sweep(args):
    """A sweep of the paper's test problems on one GPU: the cavity of Sec. 6.3 (n = 80 2^j,
    kappa = 2 pi n / 10) or the lens of Sec. 6.2 (n = 320 2^j, kappa = 300), 100-point
    leaves; one warm-up and `--steps` timed build + solve steps of the mixed path; build
    and solve timed separately with CUDA events.  One JSON line."""
    import torch

    import paper_2007_12718_gb300 as ls

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    PREC = {"fp32": ls.LS_FP32, "tf32x3": ls.LS_TF32X3, "fp16split": ls.LS_FP16SPLIT, "fp64": ls.LS_FP64}[args.precision]
    rows = []
    lens = args.sweep == "lens"
    for j in range(args.sweep_first, min(args.sweep_levels, 4) if lens else args.sweep_levels):
        name = f"lens_n{320 << j}" if lens else f"cavity_n{80 << j}"
        n, kappa, b, w = workload(name)
        h = 1.0 / n
        bd = torch.from_numpy(b).to(dev)
        f = torch.zeros(n, n, dtype=torch.complex128, device=dev)
        sig = torch.zeros_like(f)
        kw = dict(leaf_side=w["leaf"], order_precond=w["order_precond"], order_matvec=w["order_matvec"],
                  precision=PREC, top_uncompressed=args.top_uncompressed, gmres_maxit=args.sweep_maxit)
        tb = ts = 0.0
        info = bi = None
        for it in range(1 + args.steps):
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            H = ls.ls_build(n, h, kappa, bd, w["eps"], **kw)
            e[1].record(stream)
            if it == 0:
                ls.ls_rhs_plane_wave(H, [0.0], f)
                torch.cuda.synchronize()
                e[1].record(stream)
            info = ls.ls_solve(H, f, sig)[0]
            e[2].record(stream)
            bi = H.info()
            ls.ls_free(H)
            torch.cuda.synchronize()
            if it > 0:
                tb += e[0].elapsed_time(e[1]) / 1e3
                ts += e[1].elapsed_time(e[2]) / 1e3
        tb /= args.steps
        ts /= args.steps
        N = n * n
        paper = ({"iterations": PAPER_LENS[N]} if N in PAPER_LENS else None) if lens else PAPER_CAVITY.get(N)
        if paper is not None and not lens:
            paper = {"t_build_s": paper[0], "t_gmres_s": paper[1], "iterations": paper[2]}
        rows.append({"workload": name, "N": N, "kappa": kappa, "t_build_s": tb, "t_solve_s": ts,
                     "mdofs": N / (tb + ts) / 1e6, "iterations": info["iterations"],
                     "resid_true": info["resid_true"], "ranks_top": bi["ranks"][1:4],
                     "factor_GB": bi["factor_bytes"] / 1e9, "pivot_fallbacks": bi["pivot_fallbacks"],
                     "probe_resid_max": bi["probe_resid_max"], "paper": paper})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del bd, f, sig
        torch.cuda.empty_cache()
    print(json.dumps({"metric": METRIC, "sweep": ("lens, kappa = 300 (Sec. 6.2)" if lens else
                                                  "cavity, 10 points per wavelength (Sec. 6.3)"), "unit": "Mdof/s",
                      "steps": args.steps, "warmup": 1, "precision": args.precision,
                      "top_levels_uncompressed": args.top_uncompressed, "rows": rows}), flush=True)


def run_kernel_case(spec):
    """One kernel family alone, for profiling (ncu) and its roofline:
    gemm:M:N:K:ENGINE[:REPS]  the merge GEMM engine of ls_cgemm_c64 (0 SIMT, 2 tf32x3,
                              3 f16x3) on seeded random complex64 operands;
    id:M:P:R                   the blocked row ID (FP32) of a seeded M x P matrix of
                              numerical rank about R (singular values 10^(-8 i / R)).
    CUDA-event timing after two warm-up calls; one JSON line."""
    import torch

    import paper_2007_12718_gb300 as ls

    torch.manual_seed(0)
    part = spec.split(":")
    dev = torch.device("cuda", 0)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    if part[0] == "gemm":
        M, N, K, eng = (int(x) for x in part[1:5])
        reps = int(part[5]) if len(part) > 5 else 5
        A = torch.randn(1, M, K, dtype=torch.complex64, device=dev)
        B = torch.randn(1, K, N, dtype=torch.complex64, device=dev)
        C = torch.zeros(1, M, N, dtype=torch.complex64, device=dev)
        for _ in range(2):
            ls.ls_cgemm_c64(eng, A, B, C)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(reps):
            ls.ls_cgemm_c64(eng, A, B, C)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out = {"case": spec, "ms": ms, "tflops_fp32_equiv": 8.0 * M * N * K / ms / 1e9,
               "bytes_min": 8.0 * (M * K + K * N + M * N)}
    elif part[0] == "id":
        M, P, R = (int(x) for x in part[1:4])
        G1 = torch.randn(M, R, dtype=torch.complex128, device=dev)
        G2 = torch.randn(R, P, dtype=torch.complex128, device=dev)
        d = torch.pow(10.0, -8.0 * torch.arange(R, device=dev, dtype=torch.float64) / R)
        A = (G1 * d) @ G2
        for _ in range(2):
            ls.ls_row_id(A, 1e-4, precision=ls.LS_FP32, method=ls.LS_ID_BLOCKED)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        k, _, _ = ls.ls_row_id(A, 1e-4, precision=ls.LS_FP32, method=ls.LS_ID_BLOCKED)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out = {"case": spec, "ms": ms, "k": k, "tflops_8mpk": 8.0 * M * P * k / ms / 1e9,
               "note": "includes the FP64 -> FP32 conversion and the copy of U to the host"}
    else:
        raise SystemExit(f"unknown kernel case {spec}")
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, help="headline workload (paper_2007_12718_gb300.inputs.WORKLOADS)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 leg (0 = skip)")
    ap.add_argument("--fp64-warmup", type=int, default=0,
                    help="untimed FP64 steps first (the mixed warm-up already loaded every shared kernel)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the host-buffer end-to-end leg")
    ap.add_argument("--fp16-steps", type=int, default=1,
                    help="timed steps of the FP16 split-product leg on the headline workload (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 256^2 and 32^2 legs")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the differentiation workload (512x512 misfit gradient)")
    ap.add_argument("--no-multiproblem", action="store_true",
                    help="skip the many-problems workload (32 problems of sides 64..192)")
    ap.add_argument("--no-multirhs", action="store_true",
                    help="skip the multi-right-hand-side workload (512x512, 256 plane waves in one block)")
    ap.add_argument("--top-uncompressed", type=int, default=1,
                    help="tree levels kept uncompressed at the top (U = I, the ID of full rank); at 2048^2 one "
                         "level and two measure alike (0.636 and 0.632 s per step, two holding 2.4 GB more "
                         "factors); 0 compresses every level")
    ap.add_argument("--kernel-case", default=None,
                    help="time one kernel family alone (gemm:M:N:K:ENGINE[:REPS] or id:M:P:R) for profiling")
    ap.add_argument("--sweep", nargs="?", const="cavity", default=None, choices=["cavity", "lens", "direct"],
                    help="run a sweep of the paper's test problems instead of the benchmark: the cavity of "
                         "Sec. 6.3 (10 points per wavelength, default), the lens of Sec. 6.2 (kappa = 300), or "
                         "the direct solver of Sec. 6.1 (Gaussian bump, eps 1e-3 .. 1e-12)")
    ap.add_argument("--sweep-levels", type=int, default=6, help="sizes of the sweep: n = 80, 160, ..., 80 2^(levels-1)")
    ap.add_argument("--sweep-first", type=int, default=0, help="first size of the sweep: n = 80 2^first")
    ap.add_argument("--sweep-eps", default=None,
                    help="direct sweep only: comma-separated tolerances (default 1e-3,1e-6,1e-9,1e-12, n <= 640); "
                         "with it, --sweep-levels 5 reaches n = 1280")
    ap.add_argument("--sweep-maxit", type=int, default=100, help="GMRES iteration limit in the sweep (memory: "
                    "(maxit + 1) N complex128 twice)")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32x3", "fp16split", "fp64"],
                    help="engine of the mixed path's merge GEMMs (FP32 storage in both); fp64 (the plain "
                         "FP64 path) only with --sweep")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.kernel_case:
        run_kernel_case(args.kernel_case)
        return
    if args.sweep == "direct":
        run_direct_sweep(args)
        return
    if args.sweep:
        run_sweep(args)
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
