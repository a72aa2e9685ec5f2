#!/usr/bin/env python
"""Benchmark: TOD samples/s of the spin-harmonic sidelobe convolution
(Galloway et al., BeyondPlanck VIII, Sect. 2.1) at LFI-like scale:
polarised T/E/B sky and beam at lmax = 1024, kmax = 16, cube on 1024 x 2048
rings, 1e8 synthetic scan pointings (32.5 Hz, 1 rpm, 85 deg opening angle).

One step = the whole hot path on one batch: cube build (spin Legendre step +
ring FFT, synth_spin_maps) and TOD evaluation (pointing sort + interpolation
with e^{ik psi} phases, interp_tod), inputs resident in HBM.  Every launch in
the step is a kernel of libsidelobe.so.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): each rank builds the (replicated) cube and evaluates its
own consecutive shard of the scan; no data-path collective (weak scaling).
The reference arm (--impl reference) times the CPU FP64 oracle on the host
cores on a bounded sample of the same workload.

Other workloads (--workload): highres (lmax 2048, kmax 32, precision variant),
detectors (22 detectors in one CUDA graph), multisky (many skies, tensor cores),
orbital (orbital dipole through the 4pi beam), psigrid (step 2 through a psi
grid), sweep (cube-build runtime against lmax).  Each prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FSAMP = 32.5
KERNELS_PER_STEP = 6   # lcontract, ringfft, bin, scan, scatter, interp
L2_BYTES = 129 * 2 ** 20


# ----------------------------------------------------------------------------- helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_t0(rank: int, n: int, fsamp: float = FSAMP) -> float:
    """Start time of rank's shard: ranks take consecutive stretches of one scan."""
    return rank * n / fsamp


def reduce_max(value: float, device=None) -> float:
    """Max over ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "power_w_max": float(max(power)), "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# Peaks for ALU-bound kernels, from unit counts and the maximum SM clock:
#   FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.2586 TFLOP/s (NVIDIA: 1.25)
#   FP32: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz = 80.55 TFLOP/s
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# TF32 tensor peak: the measured bf16 burst (MEASURED_PEAKS.json) x the nominal TF32 / BF16 ratio (1.1 / 2.25)
PEAK_TF32_TFLOPS = measured_peaks().get("bf16_tflops", 1900.0) * 1.1 / 2.25
DTYPE = {"fp64": "f64", "fp32": "f32 (FP64 seeds/coords/final sum)",
         "df64": "f32x2 double-float contraction and interpolation (FP64 seeds/tables/FFT/coords)",
         "tf32x3": "f32 with a 3xTF32 tensor-core contraction (FP64 seeds/coords/final sum)"}
PEAK_FP32_TINST = 152 * 128 * 2.07e9 / 1e12          # FP32-pipe instructions per second (x 1e12)


# FP32 instructions per recurrence step of the double-float contraction
# (k_lcontract.cu): four double-float multiply-accumulates (12 each) and two
# fused double-float a b + c (15 each: a' x -+ b', then t y_l - y_{l-1}).
DF_LC_INST_PER_STEP = 4 * 12 + 2 * 15


def df_interp_inst(K, p=4):
    """FP32 instructions the double-float interpolation executes per sample
    (counted from k_interp_df.cu): a double-float multiply-accumulate is 12
    instructions (product with its FMA error terms, two_sum, two adds); per
    k >= 1 there are 2 p^2 of them, 2 for the phase, two normalisations (6)
    and a fused double-float Chebyshev step for cos and sin (2 x 15); k = 0
    has p^2; the weights take ~320."""
    return 12 * p * p + K * (12 * 2 * p * p + 6 + 24 + 30) + 320


def algorithmic_flops(L, K, R, n, p=4):
    """Per-launch algorithmic work (dense triangular count):
    spin Legendre step: (K+1) [4 R (L+1)^2 (complex x real MACs) + 3 R (L+1)(L+2)/2 (recurrence)];
    interpolation: n [4 p^2 (K+1) + 10]."""
    lcontract = (K + 1) * (4.0 * R * (L + 1) ** 2 + 3.0 * R * (L + 1) * (L + 2) / 2.0)
    interp = n * (4.0 * p * p * (K + 1) + 10.0)
    return lcontract, interp


# ----------------------------------------------------------------------------- GPU arm
def workload_config(cfg, n, prec, highres):
    """The `config` object of the headline workload (the same keys in both arms)."""
    L, K = cfg["lmax"], cfg["kmax"]
    R, nphi = cfg["ring_theta"].size, cfg["nphi"]
    if highres:
        workload = ("precision variant: unpolarised, lmax=%d, kmax=%d, %d rings x %d phi, %d uniform pointings "
                    "per GPU" % (L, K, R, nphi, n))
    else:
        workload = ("LFI-like: polarised T/E/B, lmax=%d, kmax=%d, %d rings x %d phi, "
                    "%d scan pointings per GPU (32.5 Hz, 1 rpm, 85 deg)" % (L, K, R, nphi, n))
    return {"workload": workload, "lmax": L, "kmax": K, "ncomp": int(cfg["sky"].shape[0]), "nrings": R, "nphi": nphi,
            "interp_order": 4, "samples_per_gpu": n, "precision": prec,
            "parallelism": "replicated cube, sharded TOD",
            "l2": "inputs larger than L2 (pointings %.1f GB, cube %.2f GB)"
                  % (24 * n / 1e9, R * nphi * (K + 1) * (16 if prec in ("fp64", "df64") else 8) / 1e9)}


def headline_metric(cfg, highres):
    if highres:
        return ("TOD samples/s (cube build+interp) at lmax=%d,kmax=%d; %%roofline; vs GPU FP64" % (cfg["lmax"], cfg["kmax"]),
                "synthetic (seeded Gaussian sky, Gaussian-taper beam, uniform pointings)")
    return ("TOD samples/s (cube build+interp) at lmax=1024,kmax=16; %roofline; vs GPU FP64",
            "synthetic (seeded T/E/B sky, far-sidelobe beam, satellite scan)")


def measure_alu(sl, device_index):
    """Measured multiply-add peaks of this GPU (sl_measure_alu_peak), TFLOP/s."""
    out = {}
    for kind in ("fp64", "fp32", "fp32x2"):
        try:
            out[kind] = round(sl.measure_alu_peak(kind, device_index) / 1e12, 4)
        except Exception as e:   # reported, not fatal
            out[kind] = None
            out["error"] = str(e)
    out["note"] = ("8 independent multiply-add chains per thread, 8 CTAs x 256 threads per SM, best of 3 (~16 ms "
                   "each); fp32x2 = packed two-lane FP32 multiply-add")
    return out


def kernel_roofs(stats, plan, prec, L, K, R, nphi, ncomp, n, alu, traffic_ok=True):
    """Rooflines of the contraction and the interpolation from one instrumented pass
    (the plan's per-kernel CUDA-event timers): algorithmic work per launch over the
    average launch time, against the peak of the unit that binds it."""
    fl_dense, fl_in = algorithmic_flops(L, K, R, n)
    lsteps = float(plan.sizes()["lsteps"])
    # the contraction skips the evanescent zone: count the work it executes,
    # 11 flops (3 recurrence + 2 complex x real MACs) per visited (ring, m, k, sign, l)
    fl_lc = 11.0 * lsteps
    suffix = {"fp64": "f64", "fp32": "f32", "df64": "df", "tf32x3": "f32"}[prec]
    lc_name = "lcontract_mma" if prec == "tf32x3" else "lcontract_" + suffix
    meas = {"fp64": alu.get("fp64"), "fp32": alu.get("fp32")}
    kernels = [
        (lc_name,
         {"fp64": fl_lc, "fp32": fl_lc, "df64": DF_LC_INST_PER_STEP * lsteps,
          # tensor work executed: 3 TF32 products x 2 flops x 16 columns (4 used, one sky)
          "tf32x3": 3 * 2.0 * 16 * lsteps}[prec],
         {"fp64": "fp64", "fp32": "fp32", "df64": "fp32inst", "tf32x3": "tf32"}[prec]),
        ("interp_" + suffix, float(n) * df_interp_inst(K) if prec == "df64" else fl_in,
         {"fp64": "fp64", "fp32": "fp32", "df64": "fp32inst", "tf32x3": "fp32"}[prec]),
    ]
    peaks = {"fp64": (PEAK_FP64_TFLOPS, "TFLOP/s", "alu", "derived: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz"),
             "fp32": (PEAK_FP32_TFLOPS, "TFLOP/s", "alu", "derived: 152 SMs x 128 FFMA/clk x 2 flops x 2.07 GHz"),
             "fp32inst": (PEAK_FP32_TINST, "Tinst/s", "alu",
                          "derived: 152 SMs x 128 FP32 instructions/clk x 2.07 GHz (double-float arithmetic)"),
             "tf32": (PEAK_TF32_TFLOPS, "TFLOP/s", "tensor",
                      "measured bf16 burst (MEASURED_PEAKS.json) x nominal TF32/BF16 ratio 1.1/2.25 (of measured)")}
    roofs = {}
    for name, work, unit_kind in kernels:
        if name not in stats or stats[name][0] <= 0:
            continue
        peak, unit, bound, note = peaks[unit_kind]
        avg_ms = stats[name][1] / stats[name][0]
        ach = work / (avg_ms / 1e3) / 1e12
        r = {"bound": bound, "achieved": round(ach, 4), "peak": round(peak, 4), "unit": unit,
             "frac": round(ach / peak, 4), "traffic": TRAFFIC.get((name, prec)) if traffic_ok else None,
             "avg_ms": round(avg_ms, 4),
             ("flops_per_launch" if unit == "TFLOP/s" else "fp32_inst_per_launch"): work, "peak_note": note}
        mp = meas.get(unit_kind)
        if mp:
            r["frac_of_measured_alu_peak"] = round(ach / mp, 4)
        roofs[name] = r
    if lc_name in roofs:
        roofs[lc_name]["flops_dense_triangle"] = fl_dense
        roofs[lc_name]["dense_equivalent_tflops"] = round(fl_dense / (roofs[lc_name]["avg_ms"] / 1e3) / 1e12, 4)
    # HBM side against the measured copy bandwidth: algorithmic bytes and (when taken
    # at this size) the ncu-measured DRAM traffic per launch over the live launch time
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
    elem = 16 if prec in ("fp64", "df64") else 8
    cube_bytes = float(R) * nphi * (K + 1) * elem
    alg_bytes = {lc_name: float(ncomp) * plan.nalm * 16 * 2 + (K + 1) * R * (2 * L + 1) * elem,
                 "interp_" + suffix: n * (8.0 + 8.0 + (24.0 if elem == 16 else 16.0) + 4.0) + cube_bytes}
    for name, r in roofs.items():
        if name in alg_bytes:
            sec = r["avg_ms"] / 1e3
            r["hbm"] = {"algorithmic_bytes": alg_bytes[name], "achieved_gbs": round(alg_bytes[name] / sec / 1e9, 1),
                        "traffic_gbs": round(r["traffic"] / sec / 1e9, 1) if r.get("traffic") else None,
                        "peak_gbs": hbm_peak, "frac": round(alg_bytes[name] / sec / 1e9 / hbm_peak, 4),
                        "note": "interpolation bytes per sample: psi 8, TOD 8, stencil record 24 (FP32 plans "
                                "16), permutation 4; plus the cube once; contraction: sky read once, G written once"}
    return roofs


def adjoint_roofs(stats, plan, K, n, alu, traffic_ok=True):
    """FP64 adjoint kernels: the interpolation transpose does the forward's
    multiply-adds per sample (4 p^2 (K+1) + 10 flops), the contraction transpose
    11 flops per (ring, m, k, sign, l) step of the forward's volume."""
    lsteps = float(plan.sizes()["lsteps"])
    out = {}
    for name, work in (("interp_adj", float(n) * (4.0 * 16 * (K + 1) + 10.0)), ("lcontract_adj", 11.0 * lsteps)):
        if name in stats and stats[name][0] > 0:
            avg_ms = stats[name][1] / stats[name][0]
            ach = work / (avg_ms / 1e3) / 1e12
            out[name] = {"bound": "alu", "achieved": round(ach, 4), "peak": round(PEAK_FP64_TFLOPS, 4),
                         "unit": "TFLOP/s", "frac": round(ach / PEAK_FP64_TFLOPS, 4), "avg_ms": round(avg_ms, 4),
                         "flops_per_launch": work, "traffic": TRAFFIC.get((name, "fp64")) if traffic_ok else None,
                         "peak_note": "derived: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz"}
            if alu.get("fp64"):
                out[name]["frac_of_measured_alu_peak"] = round(ach / alu["fp64"], 4)
    return out


def timed_steps(step, steps, stream, device, e0, e1):
    """Device time of `steps` calls of step() (CUDA events on the launching stream),
    max over ranks."""
    import torch
    barrier(device)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return reduce_max(e0.elapsed_time(e1), device)


def split_pass(plan, step, steps):
    """Per-kernel times from an instrumented pass (each launch bracketed by CUDA
    events on the plan's stream), separate from any timed region."""
    import torch
    torch.cuda.synchronize()
    plan.enable_timing(True)
    plan.kernel_stats(reset=True)
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    stats = plan.kernel_stats(reset=True)
    plan.enable_timing(False)
    return stats


def multisky_leg(sl, cfg, nsky, steps, warmup, device, local):
    """Cube builds of nsky T/E/B skies sharing the beam on the tensor cores
    (synth_spin_maps_multi, FP32 plan), with the contraction's tensor roofline."""
    import torch
    import workloads as W
    L, K, rt, nphi = cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"]
    skies = torch.from_numpy(np.stack([W.sky_polarised(L, seed=s) for s in range(nsky)])).to(device)
    beam = torch.from_numpy(cfg["beam"]).to(device)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=3, precision="fp32", device=local)
    maps = torch.empty((nsky,) + plan.maps_shape(), dtype=torch.complex64, device=device)
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step = lambda: sl.synth_spin_maps_multi(plan, skies, beam, maps)
    for _ in range(warmup):
        step()
    ms = timed_steps(step, steps, stream, device, e0, e1) / steps
    stats = split_pass(plan, step, 2)
    plan.sync()
    mma = stats.get("lcontract_mma", (1, 0.0))
    mma_ms = mma[1] / max(1, mma[0])
    nsg = (min(32, nsky) + 3) // 4 * 4
    n_cols = 4 * nsg * ((nsky + nsg - 1) // nsg)
    mma_flops = 3 * 2.0 * float(plan.sizes()["lsteps"]) * n_cols
    out = {"value": nsky / (ms / 1e3), "unit": "cubes/s", "nsky": nsky, "ms_per_step": ms, "steps": steps,
           "kernel_ms_per_step": {k: round(v[1] / 2, 4) for k, v in stats.items()}}
    if mma_ms > 0:
        ach = mma_flops / (mma_ms / 1e3) / 1e12
        out["roofline"] = {"bound": "tensor", "kernel": "lcontract_mma", "achieved": round(ach, 3),
                           "peak": round(PEAK_TF32_TFLOPS, 1), "unit": "TFLOP/s",
                           "frac": round(ach / PEAK_TF32_TFLOPS, 4), "traffic": None, "avg_ms": round(mma_ms, 4),
                           "tf32_flops_per_launch": mma_flops, "algorithmic_fp32_tflops": round(ach / 3, 3),
                           "peak_note": "measured bf16 burst x nominal TF32/BF16 ratio 1.1/2.25 (of measured); "
                                        "achieved counts 3 TF32 products x 2 flops per visited (ring pair, m, k, "
                                        "sign, l) step and column"}
    sl.plan_destroy(plan)
    del skies, maps
    torch.cuda.empty_cache()
    return out


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_2201_03478_gb300 as sl
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")

    n = int(args.n)
    highres = args.workload == "highres"
    cfg = W.config_highres(with_pointings=False) if highres else W.config_lfi(with_pointings=False)
    small = bool(args.lmax or args.nrings or args.nphi)
    # the stored DRAM traffic per launch holds for the LFI-like workload at 1e8 pointings only
    traffic_sized = not (highres or small) and n == int(1e8)
    if small:   # smaller variants of the same workload (profiling)
        Ls = args.lmax or cfg["lmax"]
        cfg = dict(cfg, lmax=Ls, sky=W.sky_polarised(Ls, seed=0), beam=W.beam_far_sidelobe(Ls, cfg["kmax"], seed=1),
                   ring_theta=W.equiangular_ring_theta(args.nrings or cfg["ring_theta"].size),
                   nphi=args.nphi or cfg["nphi"])
    L, K = cfg["lmax"], cfg["kmax"]
    ncomp = cfg["sky"].shape[0]
    rt, nphi = cfg["ring_theta"], cfg["nphi"]
    R = rt.size
    if highres:
        th, ph, ps = W.pointings_uniform(n, seed=2 + rank)
    else:
        th, ph, ps = W.pointings_scan(n, t0=shard_t0(rank, n))
    sky_h = torch.from_numpy(cfg["sky"])
    beam_h = torch.from_numpy(cfg["beam"])
    ptg_h = [torch.from_numpy(a) for a in (th, ph, ps)]
    sky = sky_h.to(device)
    beam = beam_h.to(device)
    theta, phi, psi = (t.to(device) for t in ptg_h)
    alu = measure_alu(sl, local) if (rank == 0 and args.alu_peaks) else {}

    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=ncomp, precision=args.precision, device=local)
    if args.tile_cols:
        plan.set_tile_cols(args.tile_cols)
    if args.fft_tile:
        plan.set_fft_tile(*(int(v) for v in args.fft_tile.split(",")))
    maps = torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device=device)
    tod = torch.empty(n, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def step():   # the whole forward in one call: the pointing sort runs beside the cube build
        sl.convolve_tod(plan, sky, beam, theta, phi, psi, maps=maps, tod=tod)

    def step_two_calls():   # the same work as two calls on one stream (per-kernel split, reference time)
        sl.synth_spin_maps(plan, sky, beam, maps)
        sl.interp_tod(plan, maps, theta, phi, psi, tod)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if not bool(torch.isfinite(tod).all()):
        raise RuntimeError("non-finite TOD")

    # ---- the timed region: K steps, no per-launch instrumentation
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    ms_total = timed_steps(step, args.steps, stream, device, e0, e1)
    clk = clocks.stop() if rank == 0 else None
    ms_step = ms_total / args.steps
    value = world * n * args.steps / (ms_total / 1e3)

    # ---- the two calls one after another, and the per-kernel split and rooflines
    # from a separate instrumented pass of them (kernels timed alone, not beside the sort)
    ms_two = timed_steps(step_two_calls, max(3, args.steps // 4), stream, device, e0, e1) / max(3, args.steps // 4)
    prec = args.precision
    stats = split_pass(plan, step_two_calls, args.split_steps)
    roofs = kernel_roofs(stats, plan, prec, L, K, R, nphi, ncomp, n, alu, traffic_ok=traffic_sized)
    dominant = max(stats.items(), key=lambda kv: kv[1][1])[0] if stats else None
    shares = {k: round(v[1] / max(1e-9, sum(x[1] for x in stats.values())), 4) for k, v in stats.items()}
    launches_per_step = sum(v[0] for v in stats.values()) / max(1, args.split_steps)

    metric, data = headline_metric(cfg, highres)
    config = workload_config(cfg, n, prec, highres)
    out = {
        "metric": metric,
        "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[prec],
        "data": data,
        "config": config,
        "tuning": {"tile_cols": plan.sizes()["tile_cols"],
                   "fft_tile": [plan.sizes()["fft_rings"], plan.sizes()["fft_korders"]]},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "step": "convolve_tod (cube build and interpolation in one call; the pointing sort on a second "
                "stream beside the cube build)",
        "two_calls": {"ms_per_step": ms_two, "steps": max(3, args.steps // 4),
                      "note": "synth_spin_maps then interp_tod on one stream: the same work without the overlap"},
        "kernel_split": {"steps": args.split_steps,
                         "note": "per-kernel times from a separate pass of the two calls with each launch bracketed "
                                 "by CUDA events; the timed region runs without them"},
        "kernel_ms_per_step": {k: round(v[1] / args.split_steps, 4) for k, v in stats.items()},
        "kernel_share": shares,
        "dominant_kernel": dominant,
        "roofline": roofs.get(dominant) if dominant in roofs else (next(iter(roofs.values())) if roofs else None),
        "roofline_kernels": roofs,
    }
    if rank == 0:
        out["clocks"] = clk
        out["alu_peaks_measured"] = alu

    # ---- adjoint (gradients of sum_i y_i c_i w.r.t. sky and beam) on the same pointings
    if args.adjoint_steps > 0:
        gs = torch.zeros_like(sky)
        gb = torch.zeros_like(beam)
        y = tod.clone()
        adj = lambda: sl.adjoint_tod_sharded(plan, theta, phi, psi, y, sky, beam, gs, gb)
        adj()   # warm (allocates scratch)
        torch.cuda.synchronize()
        # each rank's stretch of the scan; the gradients summed over ranks (one all-reduce)
        ms_adj = timed_steps(adj, args.adjoint_steps, stream, device, e0, e1) / args.adjoint_steps
        st_adj = split_pass(plan, adj, 1)
        out["adjoint"] = {"value": world * n / (ms_adj / 1e3), "unit": "samples/s", "ms_per_step": ms_adj,
                          "steps": args.adjoint_steps, "precision": "df64" if prec == "df64" else "fp64",
                          "kernel_ms_per_step": {k: round(v[1], 4) for k, v in st_adj.items()}}
        if prec != "df64":
            out["adjoint"]["roofline_kernels"] = adjoint_roofs(st_adj, plan, K, n, alu,
                                                               traffic_ok=traffic_sized)
        del gs, gb, y

    # ---- the other precisions on the same GPU, compared with this run's TOD
    others = [q for q in ("fp64", "df64", "fp32", "tf32x3") if q != prec] if (args.compare and rank == 0 and world == 1) else []
    out["other_precisions"] = []
    for other in others:
        p2 = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=ncomp, precision=other, device=local)
        maps2 = torch.empty(p2.maps_shape(), dtype=p2.maps_dtype, device=device)
        tod2 = torch.empty(n, dtype=torch.float64, device=device)

        def step2():
            sl.convolve_tod(p2, sky, beam, theta, phi, psi, maps=maps2, tod=tod2)

        def step2_two_calls():
            sl.synth_spin_maps(p2, sky, beam, maps2)
            sl.interp_tod(p2, maps2, theta, phi, psi, tod2)
        for _ in range(args.warmup):
            step2()
        ms2 = timed_steps(step2, args.steps, stream, device, e0, e1) / args.steps
        st2 = split_pass(p2, step2_two_calls, args.split_steps)
        err = float(torch.linalg.vector_norm(tod2 - tod) / torch.linalg.vector_norm(tod))
        out["other_precisions"].append({
            "precision": other, "dtype": DTYPE[other], "value": n / (ms2 / 1e3), "unit": "samples/s",
            "ms_per_step": ms2, "rate_vs_%s" % prec: ms_step / ms2, "tod_rel_l2_vs_%s" % prec: err,
            "kernel_ms_per_step": {k: round(v[1] / args.split_steps, 4) for k, v in st2.items()},
            "roofline_kernels": kernel_roofs(st2, p2, other, L, K, R, nphi, ncomp, n, alu,
                                             traffic_ok=traffic_sized)})
        sl.plan_destroy(p2)
        del maps2, tod2, p2
        torch.cuda.empty_cache()

    # ---- many skies with one beam on the tensor cores (the posterior-sample workload)
    if args.multisky_leg > 0 and rank == 0 and world == 1 and not highres:
        out["multisky"] = multisky_leg(sl, cfg, args.multisky_leg, max(3, args.steps // 2), args.warmup, device, local)

    # ---- end to end from pinned host buffers through the C-ABI call convolve_tod_host
    # (binding tod_from_host): copies, cube build, interpolation and download inside
    if args.e2e_steps > 0:
        pin = [t.pin_memory() for t in (sky_h, beam_h, *ptg_h)]
        res = torch.empty(n, dtype=torch.float64, pin_memory=True)   # reused TOD buffer
        torch.cuda.synchronize()
        sl.tod_from_host(plan, *pin, out=res)   # warm
        barrier(device)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sl.tod_from_host(plan, *pin, out=res)
        dt = reduce_max(time.perf_counter() - t0, device)
        h2d = sum(t.numel() * t.element_size() for t in pin)
        out["e2e"] = {"value": world * n * args.e2e_steps / dt, "unit": "samples/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(res.numel() * 8),
                      "steps": args.e2e_steps, "call": "convolve_tod_host (host buffers, 8 pieces)"}
        del pin, res

    if rank == 0 and world == 1 and args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, th, ph, ps, n, args)
    elif rank == 0:
        out["cpu_baseline"] = None
    sl.plan_destroy(plan)
    if rank == 0:
        line = json.dumps(out)
        print(line, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(line + "\n")
    if world > 1:
        dist.destroy_process_group()


def detectors_arm(args):
    """Many detectors (uneven lmax, kmax, grids and sample counts): called one by
    one, as one CUDA graph of their per-stage launches, and (FP32 plans) as the
    persistent batch -- persistent contraction and interpolation launches over
    all detectors (one per number of contraction ring pairs per thread among
    them), in one CUDA graph (sl_batch_*, SL_BATCH_PERSISTENT).  `value` is the
    faster of the two batch forms, named in `metric` and `form`."""
    import torch

    import paper_2201_03478_gb300 as sl
    import workloads as W

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dets = W.config_detectors(ndet=args.ndet)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    items = []
    for d in dets:
        plan = sl.sidelobe_plan_create(d["lmax"], d["kmax"], d["ring_theta"], d["nphi"], ncomp=3,
                                       precision=args.precision, device=local)
        items.append(dict(plan=plan, sky=dev(d["sky"]), beam=dev(d["beam"]),
                          maps=torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device=device),
                          theta=dev(d["theta"]), phi=dev(d["phi"]), psi=dev(d["psi"]),
                          tod=torch.empty(d["n"], dtype=torch.float64, device=device)))
        del d["theta"], d["phi"], d["psi"]
    ntot = sum(d["n"] for d in dets)
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def serial():
        for it in items:
            sl.synth_spin_maps(it["plan"], it["sky"], it["beam"], it["maps"])
            sl.interp_tod(it["plan"], it["maps"], it["theta"], it["phi"], it["psi"], it["tod"])

    def timed(fn, stats_on=False):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if stats_on:   # the plan's kernel timers cover the timed calls only
            plan.enable_timing(True)
            plan.kernel_stats(reset=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    # clocks sampled over every timed leg (serial, graph, persistent)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_serial = timed(serial)
    ref = [it["tod"].clone() for it in items]
    t0 = time.perf_counter()
    batch = sl.sl_batch_create(items, autotune=args.autotune)
    t_create = time.perf_counter() - t0
    ms_graph = timed(batch.run)
    identical = all(bool(torch.equal(it["tod"], r)) for it, r in zip(items, ref))
    info = batch.info()
    sl.sl_batch_destroy(batch)
    persistent = None
    if args.precision == "fp32":
        # the persistent form: persistent contraction and interpolation launches over all detectors
        t0 = time.perf_counter()
        pbatch = sl.sl_batch_create(items, autotune=args.autotune, persistent=True)
        t_pcreate = time.perf_counter() - t0
        ms_p = timed(pbatch.run)
        pbatch.sync()
        pinfo = pbatch.info()
        p_identical = all(bool(torch.equal(it["tod"], r)) for it, r in zip(items, ref))
        persistent = {"ms_per_step": ms_p, "value": ntot / (ms_p / 1e3), "create_s": t_pcreate,
                      "tuned_ms": pinfo["tuned_ms"], "kernel_nodes": pinfo["kernel_nodes"],
                      "graph_nodes": pinfo["graph_nodes"], "tod_identical_to_serial": p_identical,
                      "tile_cols": items[0]["plan"].sizes()["tile_cols"],
                      "contraction_pairs": [it["plan"].sizes()["contraction_pairs"] for it in items],
                      "fft_tile": [[it["plan"].sizes()["fft_rings"], it["plan"].sizes()["fft_korders"]] for it in items],
                      "note": "persistent k_lcontract_f32_batch launches (one per ring-pairs variant) and "
                              "k_interp_f32_cells launches (one per variant group), FFTs and sorts on branches"}
        sl.sl_batch_destroy(pbatch)
    clk = clocks.stop()
    use_p = persistent is not None and persistent["ms_per_step"] < ms_graph
    ms = persistent["ms_per_step"] if use_p else ms_graph
    form = "persistent contraction and interpolation launches in a CUDA graph" if use_p \
        else "one CUDA graph of per-detector launches"
    out = {
        "metric": "TOD samples/s (cube build+interp), %d detectors of uneven lmax/kmax, %s" % (len(dets), form),
        "value": ntot / (ms / 1e3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "form": "persistent" if use_p else "graph",
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision],
        "data": "synthetic (T/E/B sky truncated per detector, per-detector far-sidelobe beams, offset scans)",
        "config": {"workload": "multi-detector batch: %d detectors, lmax in {256..1500}, kmax in {4..24}, "
                               "%d samples in total" % (len(dets), ntot),
                   "detectors": [{"lmax": d["lmax"], "kmax": d["kmax"], "n": d["n"]} for d in dets],
                   "precision": args.precision, "autotune": bool(args.autotune),
                   "l2": "inputs larger than L2 (pointings %.1f GB)" % (24 * ntot / 1e9)},
        "serial": {"value": ntot / (ms_serial / 1e3), "ms_per_step": ms_serial,
                   "note": "the same detectors called one after another on one stream"},
        "graph": {"value": ntot / (ms_graph / 1e3), "ms_per_step": ms_graph, "nstreams": info["nstreams"],
                  "kernel_nodes": info["kernel_nodes"], "graph_nodes": info["graph_nodes"], "create_s": t_create,
                  "tuned_ms": info["tuned_ms"], "tuner_serial_ms": info["serial_ms"],
                  "tod_identical_to_serial": identical,
                  "note": "every detector's own launches in one CUDA graph, spread over parallel branches"},
        "persistent": persistent,
        "gpu_launches": persistent["kernel_nodes"] if use_p else info["kernel_nodes"],
        "clocks": clk,
    }
    line = json.dumps(out)
    print(line, flush=True)
    if args.json_out:
        with open(args.json_out, "w") as f:
            f.write(line + "\n")


def multisky_arm(args):
    """Cube builds of many skies sharing one beam (FP32 plan, LFI-like sizes):
    synth_spin_maps_multi (tensor-core contraction) against the same skies one
    by one through synth_spin_maps (CUDA-core contraction)."""
    import torch

    import paper_2201_03478_gb300 as sl
    import workloads as W

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    cfg = W.config_lfi(with_pointings=False)
    if args.lmax or args.nrings or args.nphi:   # smaller variants of the same workload (profiling)
        Ls = args.lmax or cfg["lmax"]
        cfg = dict(cfg, lmax=Ls, beam=W.beam_far_sidelobe(Ls, cfg["kmax"], seed=1),
                   ring_theta=W.equiangular_ring_theta(args.nrings or cfg["ring_theta"].size),
                   nphi=args.nphi or cfg["nphi"])
    L, K, rt, nphi = cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"]
    nsky = args.nsky
    skies = torch.from_numpy(np.stack([W.sky_polarised(L, seed=s) for s in range(nsky)])).to(device)
    beam = torch.from_numpy(cfg["beam"]).to(device)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=3, precision="fp32", device=local)
    maps = torch.empty((nsky,) + plan.maps_shape(), dtype=torch.complex64, device=device)
    one = torch.empty(plan.maps_shape(), dtype=torch.complex64, device=device)
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, stats_on=False):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if stats_on:   # the plan's kernel timers cover the timed calls only
            plan.enable_timing(True)
            plan.kernel_stats(reset=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def singles():
        for s in range(nsky):
            sl.synth_spin_maps(plan, skies[s], beam, one)

    ms_single = timed(singles)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_multi = timed(lambda: sl.synth_spin_maps_multi(plan, skies, beam, maps), stats_on=True)
    clk = clocks.stop()
    stats = plan.kernel_stats(reset=True)
    plan.enable_timing(False)
    plan.sync()
    errs = []
    for s in (0, nsky - 1):
        sl.synth_spin_maps(plan, skies[s], beam, one)
        errs.append(float(torch.linalg.vector_norm(maps[s] - one) / torch.linalg.vector_norm(one)))
    mma = stats.get("lcontract_mma", (1, 0.0))
    mma_ms = mma[1] / max(1, mma[0])
    # dense tile work the tensor cores execute per launch: three TF32 products of
    # (128 rows x N columns x 32 l) per CTA chunk; counted from the plan's recurrence volume
    nsg = min(32, nsky)
    nsg = (nsg + 3) // 4 * 4
    n_cols = 4 * nsg * ((nsky + nsg - 1) // nsg)
    mma_flops = 3 * 2.0 * float(plan.sizes()["lsteps"]) * n_cols
    out = {
        "metric": "sky cubes/s (lmax=1024, kmax=16, T/E/B, 1024x2048), %d skies sharing one beam" % nsky,
        "value": nsky / (ms_multi / 1e3), "unit": "cubes/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_multi, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (3xTF32 tensor-core contraction, FP32 accumulation)",
        "data": "synthetic (seeded T/E/B skies, far-sidelobe beam)",
        "config": {"workload": "multi-sky cube build, %d skies" % nsky, "lmax": L, "kmax": K, "nrings": rt.size,
                   "nphi": nphi, "precision": "fp32"},
        "single_sky_path": {"value": nsky / (ms_single / 1e3), "ms_per_step": ms_single,
                            "note": "synth_spin_maps once per sky (CUDA-core contraction)"},
        "speedup_vs_single_sky_path": ms_single / ms_multi,
        "cube_rel_l2_vs_single_sky_path": errs,
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in stats.items()},
        "tensor": {"kernel": "k_lcontract_mma", "avg_ms": mma_ms,
                   "tf32_flops_per_launch": mma_flops,
                   "achieved_tflops": mma_flops / (mma_ms / 1e3) / 1e12 if mma_ms > 0 else None,
                   "note": "dense TF32 work of the visited (ring, m, k, sign, l) volume; the zero rows of "
                           "not-yet-started rings inside a chunk are executed too"},
        "gpu_launches": int(sum(v[0] for v in stats.values()) / args.steps),
        "clocks": clk,
    }
    if mma_ms > 0:
        # dominant kernel against the TF32 tensor peak: the executed TF32 work (three
        # products per FP32 product) and, beside it, the FP32-equivalent algorithmic rate
        ach = mma_flops / (mma_ms / 1e3) / 1e12
        out["roofline"] = {"bound": "tensor", "kernel": "lcontract_mma", "achieved": round(ach, 3),
                           "peak": round(PEAK_TF32_TFLOPS, 1), "unit": "TFLOP/s",
                           "frac": round(ach / PEAK_TF32_TFLOPS, 4), "traffic": None, "avg_ms": round(mma_ms, 4),
                           "algorithmic_fp32_tflops": round(ach / 3, 3),
                           "peak_note": "measured bf16 burst x nominal TF32/BF16 ratio (of measured); achieved "
                                        "counts 3 TF32 products x 2 flops per visited (ring pair, m, k, sign, l) "
                                        "step and column"}
    sl.plan_destroy(plan)
    print(json.dumps(out), flush=True)


# ncu-measured DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
# at full size for the current kernels (profiles/launches_lfi_*.txt).
TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum per launch, LFI-like workload, 1e8 pointings
    # (profiles/launches_lfi_{fp64,fp32,df64}.txt; single-pass ncu metrics of the current kernels)
    ("lcontract_f64", "fp64"): 673.9e6 + 516.4e6,
    ("interp_f64", "fp64"): 15153.3e6 + 1911.1e6,
    ("lcontract_f32", "fp32"): 370.3e6 + 233.7e6,
    ("interp_f32", "fp32"): 7086.2e6 + 2115.9e6,
    ("lcontract_df", "df64"): 672.3e6 + 511.3e6,
    ("interp_df", "df64"): 22934.1e6 + 2736.6e6,
    ("interp_adj", "fp64"): 18463.7e6 + 385.5e6,
    ("lcontract_adj", "fp64"): 1507.2e6 + 285.3e6,
}


# ----------------------------------------------------------------------------- psi-grid variant
def psigrid_arm(args):
    """Step 2 as the paper states it: the transform over k to a psi grid and
    Lagrange interpolation in theta, phi and psi, against the exact phase sum
    (same plan, cube and pointings)."""
    import torch
    import torch.distributed as dist

    import paper_2201_03478_gb300 as sl
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    n = int(args.n)
    cfg = W.config_lfi(with_pointings=False)
    L, K, rt, nphi = cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"]
    npsi = args.npsi or 2 * K + 2
    th, ph, ps = W.pointings_scan(n, t0=shard_t0(rank, n))
    ptg_h = [torch.from_numpy(a) for a in (th, ph, ps)]
    theta, phi, psi = (t.to(device) for t in ptg_h)
    sky = torch.from_numpy(cfg["sky"]).to(device)
    beam = torch.from_numpy(cfg["beam"]).to(device)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=3, precision=args.precision, device=local)
    maps = torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device=device)
    rdt = torch.float64 if plan.maps_dtype == torch.complex128 else torch.float32
    cube_psi = torch.empty((rt.size, nphi, npsi), dtype=rdt, device=device)
    tod = torch.empty(n, dtype=torch.float64, device=device)
    tod_x = torch.empty(n, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)

    def step():
        sl.synth_spin_maps(plan, sky, beam, maps)
        sl.synth_psi_cube(plan, maps, npsi, cube_psi)
        sl.interp_tod_psi(plan, cube_psi, theta, phi, psi, tod)

    def step_exact():
        sl.synth_spin_maps(plan, sky, beam, maps)
        sl.interp_tod(plan, maps, theta, phi, psi, tod_x)

    def timed(fn, steps, stats_on=False):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if stats_on:
            plan.enable_timing(True)
            plan.kernel_stats(reset=True)
        barrier(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return reduce_max(e0.elapsed_time(e1), device) / steps

    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    ms_step = timed(step, args.steps, stats_on=True)
    clk = clocks.stop() if rank == 0 else None
    stats = plan.kernel_stats(reset=True)
    plan.enable_timing(False)
    ms_exact = timed(step_exact, max(1, min(args.steps, 3)))
    err = float(torch.linalg.vector_norm(tod - tod_x) / torch.linalg.vector_norm(tod_x))
    prec = args.precision
    wide = prec in ("fp64", "df64")
    P = 4
    roofs = {}
    nm = "interp_psi_f64" if wide else "interp_psi_f32"
    peak = PEAK_FP64_TFLOPS if wide else PEAK_FP32_TFLOPS
    if nm in stats and stats[nm][0] > 0:
        # p^3 weighted terms, the p^2 and p partial sums and weight products: 2 (p^3 + p^2 + p) flops a sample
        fl = 2.0 * (P ** 3 + P ** 2 + P) * n
        avg = stats[nm][1] / stats[nm][0]
        ach = fl / (avg / 1e3) / 1e12
        roofs[nm] = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                     "frac": round(ach / peak, 4), "traffic": None, "avg_ms": round(avg, 4), "flops_per_launch": fl,
                     "peak_note": "unit counts x 2.07 GHz max SM clock"}
    nc = "psi_cube_f64" if wide else "psi_cube_f32"
    if nc in stats and stats[nc][0] > 0:
        fl = 4.0 * rt.size * nphi * npsi * (K + 1)
        avg = stats[nc][1] / stats[nc][0]
        ach = fl / (avg / 1e3) / 1e12
        roofs[nc] = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                     "frac": round(ach / peak, 4), "traffic": None, "avg_ms": round(avg, 4), "flops_per_launch": fl,
                     "peak_note": "unit counts x 2.07 GHz max SM clock"}
    dominant = max(stats.items(), key=lambda kv: kv[1][1])[0] if stats else None
    out = {
        "metric": "TOD samples/s via the psi-grid cube (cube build + psi transform + 3-D interp) at "
                  "lmax=%d,kmax=%d; vs exact phase sum" % (L, K),
        "value": world * n / (ms_step / 1e3), "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE.get(prec, prec),
        "data": "synthetic (seeded T/E/B sky, far-sidelobe beam, satellite scan)",
        "config": {"workload": "psi-grid variant: LFI-like T/E/B, lmax=%d, kmax=%d, %d rings x %d phi, npsi=%d, "
                               "%d scan pointings per GPU" % (L, K, rt.size, nphi, npsi, n),
                   "npsi": npsi, "precision": prec, "l2": "inputs larger than L2"},
        "roofline": roofs.get(dominant), "roofline_all": roofs, "dominant_kernel": dominant,
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in stats.items()},
        "exact_phase_sum": {"value": world * n / (ms_exact / 1e3), "ms_per_step": ms_exact},
        "speedup_vs_exact_phase_sum": ms_exact / ms_step,
        "tod_rel_l2_vs_exact_phase_sum": err,
        "gpu_launches": int(sum(v[0] for v in stats.values()) / args.steps),
        "clocks": clk,
        "cpu_baseline": None,
    }
    sl.plan_destroy(plan)
    if rank == 0:
        line = json.dumps(out)
        print(line, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(line + "\n")
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- runtime sweep
SWEEP = [(256, 0), (256, 10), (512, 0), (512, 10), (1024, 0), (1024, 10), (2048, 0), (2048, 10), (4096, 0),
         (4096, 10), (8192, 0), (8192, 10), (512, 100)]


def sweep_arm(args):
    """Cube-build runtime against lmax (the paper's Fig. speed): random sky, an
    elliptical-Gaussian-like beam with kmax (the paper's m_max) 0 or 10, lmax 256 ... 8192
    on lmax equiangular rings x 2 lmax phi, plus the stored sidelobe models' lmax 512 /
    kmax 100.  Each point: plan creation, then synth_spin_maps timed on the device."""
    import torch

    import paper_2201_03478_gb300 as sl
    import workloads as W

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream(device)
    precs = [x for x in args.sweep_precisions.split(",") if x]
    points = []
    for L, K in SWEEP:
        if L > args.sweep_max:
            continue
        R, nphi = L, 2 * L
        rt = W.equiangular_ring_theta(R)
        ell = np.arange(L + 1, dtype=np.float64)
        sky = torch.from_numpy(W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=0)).to(device)
        beam = torch.from_numpy(W.beam_elliptical(L, K)).to(device)
        for prec in precs:
            t0 = time.perf_counter()
            plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision=prec, device=local)
            torch.cuda.synchronize()
            t_plan = time.perf_counter() - t0
            maps = torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device=device)
            steps = 3 if L <= 2048 else 1
            sl.synth_spin_maps(plan, sky, beam, maps)
            torch.cuda.synchronize()
            plan.enable_timing(True)
            plan.kernel_stats(reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                sl.synth_spin_maps(plan, sky, beam, maps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            stats = plan.kernel_stats(reset=True)
            plan.enable_timing(False)
            lsteps = float(plan.sizes()["lsteps"])
            dense = 4.0 * R * (L + 1) ** 2 * (K + 1) + 3.0 * R * (L + 1) * (L + 2) / 2 * (K + 1)
            lc = [v for k, v in stats.items() if k.startswith("lcontract")]
            lc_ms = lc[0][1] / max(1, lc[0][0]) if lc else None
            pt = {"lmax": L, "kmax": K, "nrings": R, "nphi": nphi, "precision": prec, "ms": round(ms, 3),
                  "plan_s": round(t_plan, 2), "dense_flops": dense, "executed_flops": 11.0 * lsteps,
                  "kernel_ms": {k: round(v[1] / steps, 3) for k, v in stats.items()}}
            if lc_ms and prec in ("fp64", "fp32"):
                peak = PEAK_FP64_TFLOPS if prec == "fp64" else PEAK_FP32_TFLOPS
                pt["lcontract_frac_of_peak"] = round(11.0 * lsteps / (lc_ms / 1e3) / 1e12 / peak, 4)
            points.append(pt)
            print("sweep lmax=%d kmax=%d %s: %.2f ms (plan %.1f s)" % (L, K, prec, ms, t_plan), file=sys.stderr,
                  flush=True)
            sl.plan_destroy(plan)
            del maps
            torch.cuda.empty_cache()
        del sky, beam
        torch.cuda.empty_cache()
    head = [p for p in points if p["precision"] == precs[0]]
    top = max(head, key=lambda p: (p["lmax"], p["kmax"])) if head else None
    out = {"metric": "cube build time (synth_spin_maps) against lmax, kmax 0 and 10 (Fig. speed sweep)",
           "value": top["ms"] if top else None, "unit": "ms", "n_gpus": 1, "steps": None, "warmup": 1,
           "ms_per_step": top["ms"] if top else None, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": precs[0],
           "data": "synthetic (seeded Gaussian sky C_l=(l+1)^-2, elliptical-Gaussian-like beam)",
           "config": {"workload": "runtime sweep: lmax %s, kmax {0, 10} and (512, 100); lmax rings x 2 lmax phi"
                                  % sorted({p["lmax"] for p in points}),
                      "value_point": {"lmax": top["lmax"], "kmax": top["kmax"]} if top else None},
           "sweep": points, "cpu_baseline": None, "gpu_launches": None}
    line = json.dumps(out)
    print(line, flush=True)
    if args.json_out:
        with open(args.json_out, "w") as f:
            f.write(line + "\n")


# ----------------------------------------------------------------------------- orbital dipole
ORB_SUBSAMPLE = 20
# FP64 flops k_orb_nodes executes per node (DADD + DMUL + 2 DFMA from an ncu op
# count of one launch, divided by the nodes): the three library sincos and the
# rotation and quadratic form of Eq. dipole_fast.
ORB_NODE_FLOPS = 152     # 65 DFMA + 22 DMUL per node (ncu op counts, 1e7-sample case)


def orbital_inputs(n, rank):
    import workloads as W
    cfg = W.config_orbital(n=n, with_pointings=False)
    th, ph, ps = W.pointings_scan(n, t0=shard_t0(rank, n))
    return cfg, th, ph, ps


def orbital_bytes(starts, n, s):
    """Algorithmic DRAM bytes of k_orb_eval: the 8-byte TOD write per sample, the
    node value and second derivative (16 B) per node, and the pointing (24 B) of
    each remainder sample evaluated exactly."""
    lens = np.diff(starts)
    nodes = np.where(lens > 0, (lens - 1) // s + 1, 0)
    rem = np.maximum(lens - 1 - s * (nodes - 1), 0) * (lens > 0)
    return 8.0 * n + 16.0 * nodes.sum() + 24.0 * rem.sum(), int(nodes.sum()), int(rem.sum())


def orbital_arm(args):
    """Orbital dipole and quadrupole through the 4pi beam (Sect. 3.3): the rotation at
    every 20th sample of each pointing period, a natural cubic spline in between,
    the remainder exact; the exact per-sample GPU evaluation and the CPU oracle
    are timed beside it."""
    import torch
    import torch.distributed as dist

    import paper_2201_03478_gb300 as sl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    n = int(args.n)
    s = ORB_SUBSAMPLE
    cfg, th, ph, ps = orbital_inputs(n, rank)
    starts, beta = cfg["period_start"], cfg["beta"]
    T0 = cfg["T0"]
    q = sl.quad_factor(cfg["nu"], T0)
    plan = sl.sidelobe_plan_create(cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"], ncomp=3,
                                   precision="fp64", device=local)
    ptg_h = [torch.from_numpy(a) for a in (th, ph, ps)]
    theta, phi, psi = (t.to(device) for t in ptg_h)
    beam = torch.from_numpy(cfg["beam"]).to(device)
    tod = torch.empty(n, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)

    def step(sub=s):
        sl.orbital_dipole_tod(plan, beam, T0, q, theta, phi, psi, starts, beta, subsample=sub, tod=tod)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if not bool(torch.isfinite(tod).all()):
        raise RuntimeError("non-finite orbital TOD")
    plan.enable_timing(True)
    plan.kernel_stats(reset=True)
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    barrier(device)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(device)
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop() if rank == 0 else None
    stats = plan.kernel_stats(reset=True)
    plan.enable_timing(False)
    ms_total = reduce_max(ms_total, device)
    ms_step = ms_total / args.steps
    value = world * n * args.steps / (ms_total / 1e3)
    ref_tod = tod.clone()

    # the exact per-sample evaluation (s = 1) on the GPU
    ex_steps = max(1, min(args.steps, 3))
    step(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(ex_steps):
        step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_exact = reduce_max(e0.elapsed_time(e1), device) / ex_steps
    exact_err = float(torch.max(torch.abs(ref_tod - tod)) / torch.max(torch.abs(tod)))

    bytes_eval, nnodes, nrem = orbital_bytes(starts, n, s)
    roofs = {}
    peaks = measured_peaks()
    if "orb_eval" in stats and stats["orb_eval"][0] > 0:
        # binding roof: FP64 (one DMUL + three DFMA per spline sample, the node flops per
        # remainder sample) ahead of HBM (the algorithmic bytes above)
        avg = stats["orb_eval"][1] / stats["orb_eval"][0]
        fl = 7.0 * (n - nrem) + ORB_NODE_FLOPS * nrem
        ach = fl / (avg / 1e3) / 1e12
        hbm = bytes_eval / (avg / 1e3) / 1e9
        roofs["orb_eval"] = {"bound": "alu", "achieved": round(ach, 4), "peak": round(PEAK_FP64_TFLOPS, 4),
                             "unit": "TFLOP/s", "frac": round(ach / PEAK_FP64_TFLOPS, 4),
                             "traffic": TRAFFIC.get(("orb_eval", "fp64")), "avg_ms": round(avg, 4),
                             "flops_per_launch": fl, "bytes_per_launch": bytes_eval,
                             "hbm_achieved_gbs": round(hbm, 1), "hbm_frac": round(hbm / peaks["hbm_gbs"], 4),
                             "peak_note": "FP64 pipe: unit counts x 2.07 GHz max SM clock; HBM: measured copy "
                                          "bandwidth (of measured)"}
    if ORB_NODE_FLOPS and "orb_nodes" in stats and stats["orb_nodes"][0] > 0:
        avg = stats["orb_nodes"][1] / stats["orb_nodes"][0]
        fl = ORB_NODE_FLOPS * nnodes
        ach = fl / (avg / 1e3) / 1e12
        roofs["orb_nodes"] = {"bound": "alu", "achieved": round(ach, 4), "peak": round(PEAK_FP64_TFLOPS, 4),
                              "unit": "TFLOP/s", "frac": round(ach / PEAK_FP64_TFLOPS, 4),
                              "traffic": TRAFFIC.get(("orb_nodes", "fp64")), "avg_ms": round(avg, 4),
                              "flops_per_launch": fl,
                              "peak_note": "FP64 pipe: unit counts x 2.07 GHz max SM clock; flops per node are "
                                           "the FP64 operations the kernel executes (rotation with its three "
                                           "sincos, and the quadratic form)"}
    dominant = max(stats.items(), key=lambda kv: kv[1][1])[0] if stats else None
    out = {
        "metric": "orbital dipole TOD samples/s (4pi beam; rotation every %dth sample + natural spline)" % s,
        "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (LFI-like far-sidelobe beam, satellite scan, Earth-orbit velocities)",
        "config": {"workload": "orbital dipole + quadrupole through the 4pi beam: %d scan samples per GPU in %d "
                               "pointing periods of 40-70 min, rotation every %d samples" % (n, starts.size - 1, s),
                   "subsample": s, "nodes": nnodes, "remainder_samples": nrem,
                   "l2": "inputs larger than L2 (3 x 8 B x n pointings)"},
        "roofline": roofs.get(dominant) if dominant in roofs else None,
        "roofline_all": roofs,
        "dominant_kernel": dominant,
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in stats.items()},
        "exact_gpu": {"value": world * n / (ms_exact / 1e3), "ms_per_step": ms_exact,
                      "note": "every sample rotated exactly (subsample = 1)"},
        "vs_gpu_exact": ms_exact / ms_step,
        "spline_vs_exact_max_rel": exact_err,
        "gpu_launches": int(sum(v[0] for v in stats.values()) / args.steps) + 1,   # + the moments kernel
        "clocks": clk,
    }
    # ---- end to end through the public API from pinned host buffers
    if args.e2e_steps > 0:
        pin = [t.pin_memory() for t in ptg_h]
        res = torch.empty(n, dtype=torch.float64, pin_memory=True)

        def e2e():
            for d, h in zip((theta, phi, psi), pin):
                d.copy_(h, non_blocking=True)
            step()
            res.copy_(tod, non_blocking=True)
            torch.cuda.synchronize()

        e2e()
        barrier(device)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e()
        dt = reduce_max(time.perf_counter() - t0, device)
        out["e2e"] = {"value": world * n * args.e2e_steps / dt, "unit": "samples/s",
                      "h2d_bytes_per_step": int(sum(t.numel() * 8 for t in pin)), "d2h_bytes_per_step": int(n * 8),
                      "steps": args.e2e_steps}
        del pin, res
    if rank == 0 and world == 1 and args.cpu_baseline:
        out["cpu_baseline"] = orbital_cpu(cfg, th, ph, ps, s, 3)
    elif rank == 0:
        out["cpu_baseline"] = None
    sl.plan_destroy(plan)
    if rank == 0:
        line = json.dumps(out)
        print(line, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(line + "\n")
    if world > 1:
        dist.destroy_process_group()


def orbital_cpu(cfg, th, ph, ps, s, nper_sample):
    """The oracle (numpy, one thread) on the first whole pointing periods."""
    from oracle import orbital as orb
    starts, beta = cfg["period_start"], cfg["beta"]
    e = int(starts[nper_sample])
    S = orb.moments(cfg["beam"][0])
    q = orb.quad_factor(cfg["nu"], cfg["T0"])
    t0 = time.perf_counter()
    orb.dipole_subsampled(S, cfg["T0"], q, th[:e], ph[:e], ps[:e], starts[:nper_sample + 1], beta[:nper_sample], s)
    dt = time.perf_counter() - t0
    return {"value": e / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": "the first %d pointing periods (%d samples), subsample %d, %.1f s" % (nper_sample, e, s, dt)}


def orbital_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = int(args.n)
    cfg, th, ph, ps = orbital_inputs(n, 0)
    for _ in range(args.warmup):
        orbital_cpu(cfg, th, ph, ps, ORB_SUBSAMPLE, 1)
    per = [orbital_cpu(cfg, th, ph, ps, ORB_SUBSAMPLE, 3) for _ in range(args.steps)]
    value = float(np.mean([p["value"] for p in per]))
    out = {"impl": "reference",
           "metric": "orbital dipole TOD samples/s (4pi beam; rotation every %dth sample + natural spline)"
                     % ORB_SUBSAMPLE,
           "value": world * value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": n / value * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (LFI-like far-sidelobe beam, satellite scan, Earth-orbit velocities)",
           "config": {"workload": "orbital dipole + quadrupole through the 4pi beam: %d scan samples per GPU, "
                                  "rotation every %d samples" % (n, ORB_SUBSAMPLE), "subsample": ORB_SUBSAMPLE},
           "cpu_baseline": dict(per[-1], value=value),
           "e2e": {"value": world * value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- CPU oracle timing
def oracle_sample(cfg, th, ph, ps, n, ring_sample, samp_n):
    """Time the CPU FP64 oracle on a bounded sample of one step and extrapolate:
    spin Legendre step + DFT for `ring_sample` of the rings, interpolation of
    `samp_n` of the n samples.  Returns (seconds per full step, detail)."""
    import oracle
    rt = cfg["ring_theta"]
    R = rt.size
    idx = np.linspace(0, R - 1, ring_sample).round().astype(int)
    t0 = time.perf_counter()
    G = oracle.cube_G(cfg["sky"], cfg["beam"], rt[idx])
    oracle.cube_from_G(G, cfg["nphi"])
    t_cube = time.perf_counter() - t0
    cube = np.zeros((R, cfg["nphi"], cfg["kmax"] + 1), dtype=np.complex128)
    t0 = time.perf_counter()
    oracle.interp(cube, rt, th[:samp_n], ph[:samp_n], ps[:samp_n])
    t_int = time.perf_counter() - t0
    full = t_cube * R / ring_sample + t_int * n / samp_n
    return full, {"cube_s": t_cube, "interp_s": t_int}


def cpu_baseline(cfg, th, ph, ps, n, args):
    rs, sn = args.cpu_rings, args.cpu_samples
    full, det = oracle_sample(cfg, th, ph, ps, n, rs, sn)
    return {"value": n / full, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "spin Legendre step + DFT on %d of %d rings, interpolation of %d of %d samples; "
                      "extrapolated to one full step (%.1f s measured)"
                      % (rs, cfg["ring_theta"].size, sn, n, det["cube_s"] + det["interp_s"])}


def reference_arm(args):
    """The oracle timed on the host cores, each step a bounded sample of the
    workload (the spin Legendre step + DFT on a subset of rings, the
    interpolation of a subset of samples).  `ms_per_step` is the time one such
    step took; `value` is the metric for the full workload, extrapolated from
    the sample (the per-ring and per-sample costs are uniform), with the
    extrapolated full-step time beside it."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads as W
    n = int(args.n)
    highres = args.workload == "highres"
    cfg = W.config_highres(with_pointings=False) if highres else W.config_lfi(with_pointings=False)
    sn = args.cpu_samples
    th, ph, ps = W.pointings_uniform(sn, seed=2) if highres else W.pointings_scan(sn)
    for _ in range(args.warmup):
        oracle_sample(cfg, th, ph, ps, n, 4, min(sn, 100000))
    per, meas = [], []
    for _ in range(args.steps):
        full, det = oracle_sample(cfg, th, ph, ps, n, args.ref_rings, sn)
        per.append(full)
        meas.append(det["cube_s"] + det["interp_s"])
    full = float(np.mean(per))
    value = world * n / full
    R = cfg["ring_theta"].size
    metric, data = headline_metric(cfg, highres)
    out = {"impl": "reference", "metric": metric,
           "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": float(np.mean(meas)) * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": data,
           "config": workload_config(cfg, n, "fp64", highres),
           "extrapolated_ms_per_full_step": full * 1e3,
           "sample_per_step": {"rings": args.ref_rings, "of_rings": R, "samples": sn, "of_samples": n},
           "cpu_baseline": {"value": value, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "each step: oracle spin Legendre step + DFT on %d of %d rings and "
                                      "interpolation of %d of %d samples (%.2f s measured per step); value "
                                      "extrapolated to the full step" % (args.ref_rings, R, sn, n, float(np.mean(meas)))},
           "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "measured_seconds": float(np.sum(meas))}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--precision", choices=["fp64", "fp32", "df64", "tf32x3"], default="fp64")
    ap.add_argument("--workload", choices=["lfi", "highres", "detectors", "multisky", "orbital", "psigrid", "sweep"],
                    default="lfi",
                    help="lfi: T/E/B, lmax 1024, kmax 16, scan (the headline); "
                         "highres: lmax 2048, kmax 32, 2048 x 4096 rings, uniform pointings (precision variant); "
                         "detectors: 22 detectors of uneven lmax/kmax in one CUDA graph (batch variant); "
                         "multisky: cubes of many skies with one beam (tensor cores); "
                         "orbital: orbital dipole through the 4pi beam; "
                         "psigrid: step 2 through a psi-grid cube, against the exact phase sum; "
                         "sweep: cube-build runtime against lmax (Fig. speed)")
    ap.add_argument("--ndet", type=int, default=22, help="detectors of the batch workload")
    ap.add_argument("--nsky", type=int, default=32, help="skies of the multi-sky workload")
    ap.add_argument("--npsi", type=int, default=0, help="psi grid of the psigrid workload (0: 2 kmax + 2)")
    ap.add_argument("--sweep-max", type=int, default=8192, help="largest lmax of the sweep workload")
    ap.add_argument("--sweep-precisions", default="fp64,fp32,df64", help="plans of the sweep workload")
    ap.add_argument("--tile-cols", type=int, default=0, help="sort-tile width (8, 16, 32; 0: the plan's default)")
    ap.add_argument("--fft-tile", default="", help="rings,korders per CTA of the ring FFT (e.g. 2,1; default: the plan's)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--n", type=float, default=0, help="pointings per GPU (default 1e8; 2e8 for highres)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--split-steps", type=int, default=3,
                    help="steps of the separate instrumented pass that gives the per-kernel split")
    ap.add_argument("--multisky-leg", type=int, default=32,
                    help="skies of the tensor-core multi-sky leg of the headline line (0: skip)")
    ap.add_argument("--no-alu-peaks", dest="alu_peaks", action="store_false",
                    help="skip the measured ALU peaks (sl_measure_alu_peak)")
    ap.add_argument("--adjoint-steps", type=int, default=3, help="timed adjoint_tod calls (0: skip)")
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-rings", type=int, default=96)
    ap.add_argument("--cpu-samples", type=int, default=8_000_000)
    ap.add_argument("--ref-rings", type=int, default=16)
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--lmax", type=int, default=0, help="override lmax (smaller profiling variants)")
    ap.add_argument("--nrings", type=int, default=0, help="override the number of equiangular rings")
    ap.add_argument("--nphi", type=int, default=0, help="override phi samples per ring")
    args = ap.parse_args(argv)
    if not args.n:
        args.n = 2e8 if args.workload == "highres" else 1e8
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, _ = dist_env()
    if world != args.gpus:
        print("note: WORLD_SIZE=%d, --gpus=%d; using WORLD_SIZE" % (world, args.gpus), file=sys.stderr)
    if args.impl == "reference" and args.workload == "orbital":
        orbital_reference(args)
    elif args.impl == "reference":
        if args.cpu_samples > 2_000_000:
            args.cpu_samples = 2_000_000
        reference_arm(args)
    elif args.workload == "orbital":
        orbital_arm(args)
    elif args.workload == "psigrid":
        psigrid_arm(args)
    elif args.workload == "sweep":
        sweep_arm(args)
    elif args.workload == "detectors":
        detectors_arm(args)
    elif args.workload == "multisky":
        multisky_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
