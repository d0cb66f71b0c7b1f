#!/usr/bin/env python
"""Benchmark of the emulator's hot path on GB300: covariance build -> adaptive
mixed-precision tile Cholesky -> emulations L z.

Workload (default): bandlimit L=128 (n = L^2 = 16384), tile nb=512, beta=8,
sigma_l = (1+l)^-1.5, nugget 1e-8; adaptive FP64/FP32/BF16 tiles at
eps = 1e-8; 256 samples, seed 1.  One "step" is the whole path on one
synthetic covariance, inputs already in HBM.  The metric is Cholesky TFLOP/s
counted as n^3/3 per step over the step time; the plain FP64 tile Cholesky of
the same matrix on the same GPU is timed beside it for the speedup.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank factors its own covariance (independent
problems, weak scaling, no collective on the data path); rank 0 prints the
JSON line with the max time over ranks.  --impl reference times the CPU
oracle (test infrastructure) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Cholesky TFLOP/s (n³/3) & speedup vs FP64 on 1 GB300 at ‖LLᵀ−Σ‖/‖Σ‖≤ε"
MASK_FP64_FP32_BF16 = 0b01011


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--nb", type=int, default=512)
    ap.add_argument("--beta", type=float, default=8.0)
    ap.add_argument("--eps", type=float, default=1e-8)
    ap.add_argument("--mask", type=int, default=MASK_FP64_FP32_BF16,
                    help="classes the norm rule may use (bit c = class c: 1 FP64, 2 FP32, 4 TF32, 8 BF16, 16 E4M3)")
    ap.add_argument("--samples", type=int, default=256)
    ap.add_argument("--seed", type=int, default=None, help="sample seed (default: 1 single, 3 batched)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--no-empirical", action="store_true", help="skip the empirical-covariance build from residuals")
    ap.add_argument("--no-bands", action="store_true", help="skip the paper's band-map variants (DP/SP, DP/SP/HP, "
                                                             "DP/HP) of the same factor")
    ap.add_argument("--workload", choices=["single", "batched", "fp64_L400"], default="single",
                    help="single: one n=L^2 covariance (default); batched: --count covariances of random "
                         "bandlimit L in [8, 64], beta in [2, 8) (SplitMix64 draws from --batch-seed)")
    ap.add_argument("--configs", default="cfg1,cfg3,cfg4,cfg5,fp64tc",
                    help="the other workloads measured beside the headline one (comma list, '' for none): "
                         "cfg1 = L=32 plain FP64; cfg3 = L=256 with E4M3 tiles and refinement; cfg4 = L=480 "
                         "class-format storage; cfg5 = the batch of 1024; fp64tc = the headline matrix with every "
                         "tile FP64-class on the tensor cores")
    ap.add_argument("--count", type=int, default=1024)
    ap.add_argument("--batch-seed", type=int, default=3)
    return ap.parse_args()


def workload_name(a) -> str:
    names = ("FP64", "FP32", "TF32", "BF16", "E4M3")
    cls = "/".join(nm for c, nm in enumerate(names) if (a.mask | 1) >> c & 1)
    return (f"L={a.L} n={a.L * a.L} nb={a.nb} beta={a.beta:g}: adaptive {cls} tile Cholesky at "
            f"eps={a.eps:g}, FP32 accumulate, + {a.samples} samples seed {a.seed}")


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    INTERVAL_MS = 50

    def start(self, ready_timeout_s: float = 3.0):
        """Starts the sampler and returns once it has written its first sample (or after ready_timeout_s), so that
        sampling runs through the whole timed region that follows."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
            return
        t_end = time.monotonic() + ready_timeout_s
        while time.monotonic() < t_end and self.proc.poll() is None:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        smax = float(parts[2])
                    except ValueError:
                        continue
                    for nm, v in zip(names, parts[5:9]):
                        if v.lower().startswith("active"):
                            reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- ours
def run_ours(a):
    import numpy as np
    import torch

    import paper_2408_04440_gb300 as E

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2408_04440_gb300 import build as _b

    if rank == 0 or world == 1:
        _b.build()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.Stream()
    ctx = E.Context(local, stream=stream)
    n, s = a.L * a.L, a.samples
    flops = n ** 3 / 3.0
    alu = {}
    try:
        f64, f32 = ctx.alu_peaks()
        alu = {"fp64_fma_tflops": round(f64, 3), "fp32_fma_tflops": round(f32, 2)}
    except Exception:  # the rooflines then fall back to the earlier probe values
        pass
    Y = E._colmajor_empty(n, s, ctx.device)
    seed = a.seed + 1000 * rank

    factor_ms = []

    def step():
        A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
        info = E.emu_potrf_mp(ctx, A, eps=a.eps, prec_mask=a.mask)
        factor_ms.append(info.ms)
        E.emu_sample(ctx, A, s, seed=seed, out=Y)
        A.free()
        return info

    with torch.cuda.stream(stream):
        # untimed setup: the library's tuner times its four reserved-SM choices
        # on the first four factors of a matrix signature (each choice's first
        # factor also records its CUDA graph); they run here, before the W
        # warm-up steps, so that every timed step uses the tuned schedule
        tuning_steps = 0
        while tuning_steps < 8 and ctx.schedule_info()[0] < 4:
            step()
            tuning_steps += 1
        for _ in range(max(a.warmup, 0)):
            info = step()
        factor_ms.clear()
        clocks = ClockSampler(local)
        barrier()
        launches0 = ctx.launch_count
        host0 = ctx.host_launch_count
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            info = step()
        e1.record(stream)
        stream.synchronize()
        barrier()
        clk = clocks.stop()
        gpu_launches = ctx.launch_count - launches0
        host_launches = ctx.host_launch_count - host0
        ms_total = e0.elapsed_time(e1)
        t = torch.tensor([ms_total], device=ctx.device)
        if dist is not None:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item()) / a.steps
        value = world * flops / (ms_per_step * 1e-3) / 1e12

        if rank != 0:
            ctx.close()
            if dist is not None:
                dist.barrier()
                dist.destroy_process_group()
            return

        mixed_factor_ms = statistics.median(factor_ms)
        _, r_free, r_free64 = ctx.schedule_info()
        extra = {"factor_ms": round(mixed_factor_ms, 4),
                 "schedule": {"tuning_steps_before_warmup": tuning_steps, "reserved_sms": r_free,
                              "reserved_sms_fp64": r_free64},
                 "factor_tflops": round(flops / (mixed_factor_ms * 1e-3) / 1e12, 3),
                 "tiles_per_class": dict(zip(E.CLASS_NAMES, info.tiles)),
                 "update_flop_share": {c: round(f / max(sum(info.update_flops), 1.0), 4)
                                       for c, f in zip(E.CLASS_NAMES, info.update_flops)}}

        # per-kernel-group device time of one profiled step (events on the launch stream)
        ctx.prof_enable(True)
        step()
        prof = ctx.prof_read()
        ctx.prof_enable(False)
        step_ms = sum(v["ms"] for v in prof.values())
        extra["kernel_groups"] = {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                      "share": round(v["ms"] / step_ms, 4)} for k, v in prof.items() if v["launches"]}
        peaks = load_peaks()
        peaks.update(alu)
        roof = roofline(prof, peaks, (a.L, a.nb, a.eps, a.mask))
        extra["measured_peaks"] = dict(alu, **tensor_peaks())

        # accuracy: backward error on 64 sampled rows against the GPU-built covariance
        extra["backward_error_rows64"] = backward_error_rows(E, ctx, a, rows=64)
        extra["backward_error_note"] = ("||(L L^T - S)[rows, :]||_F / ||S[rows, :]||_F over 64 sampled rows, S the "
                                        "GPU-built covariance; the full backward error against the oracle's S is "
                                        "checked in tests/test_gpu_full_size.py")

        if not a.no_fp64:
            A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
            E.emu_potrf_mp(ctx, A)  # warm-up of the FP64 path
            A.free()
            A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
            i64 = E.emu_potrf_mp(ctx, A)
            A.free()
            extra["fp64_factor_ms"] = round(i64.ms, 3)
            extra["fp64_tflops"] = round(flops / (i64.ms * 1e-3) / 1e12, 4)
            extra["speedup_vs_fp64"] = round(i64.ms / mixed_factor_ms, 2)
            extra["cusolver_dpotrf"] = cusolver_reference(E, ctx, a, flops)

        if not a.no_bands:
            extra["band_maps"] = band_variants(E, ctx, a, flops, extra.get("fp64_factor_ms"))
            extra["tf32_variant"] = tf32_variant(E, ctx, a, flops, extra.get("fp64_factor_ms"))
        if not a.no_empirical:
            extra["empirical_cov"] = empirical_variant(E, ctx, a)
            extra["emulation"] = emulation_variant(E, ctx, a)

        e2e = None if a.no_e2e else run_e2e(E, ctx, a, flops)
        if a.configs:
            extra["configs"] = other_configs(E, ctx, a, flops, mixed_factor_ms)

    cpu = None if (a.no_cpu or world > 1) else cpu_baseline(a)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed:f64+f32(3xbf16 split)+bf16", "data": "synthetic",
        "config": {"workload": workload_name(a), "L": a.L, "n": n, "nb": a.nb, "beta": a.beta, "eps": a.eps,
                   "samples": s, "seed": a.seed, "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2: each step rebuilds the 1.1 GB FP64 tile arena"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
        "host_launches_per_step": round(host_launches / a.steps, 1), "clocks": clk,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture of the current kernel code, keyed by (group, L, nb, eps, mask) of the
# captured workload (profiles/k_tc_gemm_L128_n16384_traffic.md: 112 launches per
# factor, 11.15 GB); None for any other workload or group.
TRAFFIC = {("tc_factor", 128, 512, 1e-8, MASK_FP64_FP32_BF16): 99.6e6}


ALU_NOTES = {
    "potrf": "the diagonal-tile POTRF is bound by its FP64 dependency chain (one 16-column leaf after another)",
    "update64": "FP64 tile updates are FP64-pipe bound; their launch times include sharing the SMs with the "
                "concurrent streams",
    "trsm64": "the FP64 panel TRSM is bound by its substitution chain and by the SMs left beside the bulk update",
    "trmm64": "FP64-class tiles of the sampler, FP64-pipe bound",
    "solve": "triangular solves, bound by their substitution chains",
    "trsm32": "the SIMT FP32 panel TRSM (tile sizes whose trailing columns do not fit in TMEM) is bound by its "
              "substitution chain and by L_kk strip loads, on the SMs left beside the bulk update",
}
# ALU peaks (TFLOP/s): measured in each run by the library's FMA-loop probe
# (emu_measure_alu_peaks: eight independent FMA chains per thread, eight CTAs of
# 256 threads per SM); these values (the same probe on a GB300) stand in only
# where the probe cannot run.
ALU_PEAK = {"fp64": 1.19, "fp32": 74.0}
ALU_GROUPS = {"potrf": "fp64", "trsm64": "fp64", "update64": "fp64", "trmm64": "fp64", "solve": "fp64",
              "trsm32": "fp32"}


def tensor_peaks() -> dict:
    """cuBLAS TF32 and FP8-E4M3 GEMM rates (8192^3, best of five, CUDA events): the measured denominators of
    the TF32 and E4M3 classes (BF16's are in MEASURED_PEAKS.json)."""
    import torch

    out = {}
    n = 8192

    def best(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        ts = []
        for _ in range(5):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return 2.0 * n ** 3 / (min(ts) * 1e-3) / 1e12

    try:
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        out["tf32_cublas_tflops"] = round(best(lambda: a @ b), 1)
        torch.backends.cuda.matmul.allow_tf32 = prev
        a8 = a.to(torch.float8_e4m3fn)
        b8 = b.to(torch.float8_e4m3fn)
        one = torch.tensor(1.0, device="cuda")
        out["e4m3_cublas_tflops"] = round(best(lambda: torch._scaled_mm(a8, b8.t(), scale_a=one, scale_b=one,
                                                                         out_dtype=torch.bfloat16)), 1)
        del a, b, a8, b8
    except Exception as exc:  # a missing library path is reported, not fatal
        out["tensor_peaks_error"] = f"{type(exc).__name__}: {exc}"
    return out


def roofline(prof: dict, peaks: dict, wl=None) -> dict:
    """Roofline of the kernel group with the largest device time in the step; wl = (L, nb, eps, mask) of the
    workload, for the DRAM traffic of its ncu capture."""
    group = max(prof, key=lambda k: prof[k]["ms"])
    g = prof[group]
    per_launch_ms = g["ms"] / max(g["launches"], 1)
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    src = "of measured" if "bf16_tflops_sustained" in peaks else "of fallback"
    if g["mma_flops"] > 0:
        # tensor cores: algorithmic flops against the precision-weighted peak of
        # this launch's class mix (FP32 class = six BF16 products)
        achieved = g["flops"] / (g["ms"] * 1e-3) / 1e12
        peak = bf16 * g["flops"] / g["mma_flops"]
        return {"kernel": group, "bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": TRAFFIC.get((group,) + tuple(wl)) if wl else None,
                "per_launch_ms": round(per_launch_ms, 4), "launches": g["launches"],
                "peak_note": f"bf16 sustained {bf16} TF/s {src}, weighted by the class mix"}
    if group in ALU_GROUPS:
        unit = ALU_GROUPS[group]
        peak = peaks.get(f"{unit}_fma_tflops") or ALU_PEAK[unit]
        psrc = "measured in this run" if f"{unit}_fma_tflops" in peaks else "of an earlier probe run"
        achieved = g["flops"] / (g["ms"] * 1e-3) / 1e12
        return {"kernel": group, "bound": "alu", "achieved": round(achieved, 4), "peak": peak, "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": TRAFFIC.get((group,) + tuple(wl)) if wl else None,
                "per_launch_ms": round(per_launch_ms, 4), "launches": g["launches"],
                "peak_note": f"{unit.upper()} FMA-loop peak {psrc}; " + ALU_NOTES.get(group, "")}
    hbm = peaks.get("hbm_gbs") or 6800.0
    achieved = g["bytes"] / (g["ms"] * 1e-3) / 1e9
    return {"kernel": group, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": None, "per_launch_ms": round(per_launch_ms, 4),
            "launches": g["launches"]}


def backward_error_rows(E, ctx, a, rows: int, band: int = 0, mask: int = MASK_FP64_FP32_BF16) -> float:
    import torch

    n = a.L * a.L
    S = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
    Sd = E.emu_mat_export(ctx, S)  # lower triangle
    S.free()
    Sd = Sd + Sd.t() - torch.diag(torch.diag(Sd))
    A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
    E.emu_potrf_mp(ctx, A, eps=a.eps, prec_mask=mask, band=band)
    Ld = E.emu_mat_export(ctx, A)
    A.free()
    g = torch.Generator().manual_seed(7)
    idx = torch.randperm(n, generator=g)[:rows].to(Ld.device)
    R = Ld[idx, :] @ Ld.t() - Sd[idx, :]
    be = float(torch.linalg.norm(R) / torch.linalg.norm(Sd[idx, :]))
    del Sd, Ld, R
    torch.cuda.empty_cache()
    return be


def band_variants(E, ctx, a, flops, fp64_ms) -> dict:
    """The paper's band-map precision variants of the same factor (diagonal band
    FP64; DP/SP: the rest FP32; DP/SP/HP: 5 % of the tiles FP32 in the bands
    next to the diagonal, the rest BF16; DP/HP: the rest BF16): factor time
    (median of two after a warm-up), class counts and the sampled-row backward
    error.  Their accuracy is what the map gives, not a requested eps."""
    out = {}
    for band in (E.MAP_DP_SP, E.MAP_DP_SP_HP, E.MAP_DP_HP):
        ts, info = [], None
        for r in range(3):
            A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
            info = E.emu_potrf_mp(ctx, A, band=band, raise_on_error=False)
            A.free()
            if info.status != E.EMU_OK:
                break
            if r:
                ts.append(info.ms)
        name = E.MAP_NAMES[band]
        if info.status != E.EMU_OK:
            out[name] = {"status": int(info.status),
                         "pivot": info.pivot}
            continue
        fms = statistics.median(ts)
        d = {"factor_ms": round(fms, 3), "tflops": round(flops / (fms * 1e-3) / 1e12, 3),
             "tiles_per_class": dict(zip(E.CLASS_NAMES, info.tiles)),
             "backward_error_rows64": backward_error_rows(E, ctx, a, rows=64, band=band)}
        if fp64_ms:
            d["speedup_vs_fp64"] = round(fp64_ms / fms, 2)
        out[name] = d
    return out


def tf32_variant(E, ctx, a, flops, fp64_ms) -> dict:
    """The same factor and eps with the TF32 class enabled beside FP64/FP32/BF16
    (tiles that pass at u = 2^-11 take one kind::tf32 product instead of six
    BF16 split products)."""
    mask = MASK_FP64_FP32_BF16 | (1 << 2)
    ts, info = [], None
    for r in range(3):
        A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
        info = E.emu_potrf_mp(ctx, A, eps=a.eps, prec_mask=mask)
        A.free()
        if r:
            ts.append(info.ms)
    fms = statistics.median(ts)
    d = {"prec_mask": mask, "factor_ms": round(fms, 3), "tflops": round(flops / (fms * 1e-3) / 1e12, 3),
         "tiles_per_class": dict(zip(E.CLASS_NAMES, info.tiles)),
         "backward_error_rows64": backward_error_rows(E, ctx, a, rows=64, mask=mask)}
    if fp64_ms:
        d["speedup_vs_fp64"] = round(fp64_ms / fms, 2)
    return d


def empirical_variant(E, ctx, a) -> dict:
    """The empirical covariance of the paper's emulator (U-hat = sum of xi xi^T
    over the residual vectors / their number) from m = n synthetic residuals
    drawn through our own sampler (xi = L z with L the mixed factor of the
    synthetic covariance), then its mixed factor at the same eps.  The build
    is the symmetric product on the tensor cores with FP64 accuracy; its
    algorithmic flops are n (n + 1) m."""
    import time
    import torch

    n = a.L * a.L
    m = n
    A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
    E.emu_potrf_mp(ctx, A, eps=a.eps, prec_mask=MASK_FP64_FP32_BF16)
    Xi = E._colmajor_empty(n, m, ctx.device)
    E.emu_sample(ctx, A, m, seed=11, out=Xi)
    A.free()
    ts, U = [], None
    for r in range(3):
        if U is not None:
            U.free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U, _ = E.emu_cov_from_residuals(ctx, Xi, nb=a.nb, nugget_rel=0.0)  # the call returns when U is built
        t1 = time.perf_counter()
        if r:
            ts.append((t1 - t0) * 1e3)
    del Xi
    torch.cuda.empty_cache()
    bms = statistics.median(ts)
    info = E.emu_potrf_mp(ctx, U, eps=a.eps, prec_mask=MASK_FP64_FP32_BF16, raise_on_error=False)
    U.free()
    d = {"residuals": m, "build_ms": round(bms, 2), "build_tflops": round(n * (n + 1) * m / (bms * 1e-3) / 1e12, 2),
         "build_note": "host wall time of the synchronous call, planning included",
         "factor_status": int(info.status), "factor_ms": round(info.ms, 3),
         "tiles_per_class": dict(zip(E.CLASS_NAMES, info.tiles))}
    return d


def emulation_variant(E, ctx, a, T: int = 256) -> dict:
    """Emulations from the mixed factor: T draws xi_t = L z_t, the VAR(3)
    recursion with diagonal Phi (0.5, 0.2, 0.1 for every coefficient), the
    inverse SHT to an (L+1) x 2L grid per time step, and the forward SHT of
    those grids back to coefficients.  Times of the calls (host wall time of
    the synchronous calls), grid points per second, round-trip error."""
    import time
    import torch

    n = a.L * a.L
    A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
    E.emu_potrf_mp(ctx, A, eps=a.eps, prec_mask=MASK_FP64_FP32_BF16)
    Xi = E._colmajor_empty(n, T, ctx.device)
    E.emu_sample(ctx, A, T, seed=12, out=Xi)
    A.free()
    Ph = torch.tensor([0.5, 0.2, 0.1], dtype=torch.float64, device=Xi.device).repeat(n, 1)
    nt, nph = a.L + 1, 2 * a.L
    tv, ti = [], []
    for r in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F = E.emu_var_recursion(ctx, Xi, Ph)
        t1 = time.perf_counter()
        Z = E.emu_isht(ctx, F, a.L, nt, nph)
        t2 = time.perf_counter()
        if r:
            tv.append((t1 - t0) * 1e3)
            ti.append((t2 - t1) * 1e3)
    ims = statistics.median(ti)
    # the forward transform of the same grids recovers the coefficients (band-limited data, ntheta = L + 1)
    tf = []
    for r in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F2 = E.emu_sht(ctx, Z, a.L, nt, nph)
        t1 = time.perf_counter()
        if r:
            tf.append((t1 - t0) * 1e3)
    rt = float((F2 - F).abs().max() / F.abs().max())
    out = {"time_steps": T, "grid": [nt, nph], "var_ms": round(statistics.median(tv), 3), "isht_ms": round(ims, 3),
           "sht_ms": round(statistics.median(tf), 3), "grid_points_per_s": round(nt * nph * T / (ims * 1e-3), 1),
           "sht_round_trip_rel_err": rt, "finite": bool(torch.isfinite(Z).all())}
    del Xi, F, Z, F2
    torch.cuda.empty_cache()
    return out


def cusolver_reference(E, ctx, a, flops) -> dict:
    """cuSOLVER's dense FP64 Cholesky (torch.linalg.cholesky) of the same
    covariance on the same GPU: an extra reference row, not our path."""
    import torch

    A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
    Sd = E.emu_mat_export(ctx, A)
    A.free()
    Sd = Sd + Sd.t() - torch.diag(torch.diag(Sd))
    ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Lc = torch.linalg.cholesky(Sd)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        del Lc
    del Sd
    torch.cuda.empty_cache()
    t = min(ms)
    return {"ms": round(t, 3), "tflops": round(flops / (t * 1e-3) / 1e12, 4),
            "call": "torch.linalg.cholesky (cuSOLVER potrf), FP64, dense n x n"}


def run_e2e(E, ctx, a, flops) -> dict:
    """Same step through the C ABI with HOST buffers: the covariance comes from
    pinned host memory (lower triangle copied tile column by tile column) and
    the samples go back to pinned host memory, copies inside the timed region."""
    import torch

    n, s, nb = a.L * a.L, a.samples, a.nb
    A = E.emu_cov_build(ctx, a.L, a.beta, nb)
    Sd = E.emu_mat_export(ctx, A)
    A.free()
    hS = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()  # column-major host
    hS.copy_(Sd)
    del Sd
    torch.cuda.empty_cache()
    hY = torch.empty((s, n), dtype=torch.float64, pin_memory=True).t()
    NT = (n + nb - 1) // nb
    h2d = sum((n - j * nb) * min(nb, n - j * nb) * 8 for j in range(NT))
    d2h = n * s * 8

    def step():
        M = E.emu_mat_import_host(ctx, hS, nb)
        E.emu_potrf_mp(ctx, M, eps=a.eps, prec_mask=MASK_FP64_FP32_BF16)
        E.emu_sample_host(ctx, M, s, seed=a.seed, out=hY)
        M.free()

    for _ in range(2):
        step()
    k = max(3, min(a.steps, 10))
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / k
    return {"value": round(flops / dt / 1e12, 4), "unit": "TFLOP/s", "ms_per_step": round(dt * 1e3, 3),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": k,
            "path": "emu_mat_import_host -> emu_potrf_mp -> emu_sample_host"}


# ------------------------------------------------------------- CPU oracle
# ------------------------------------------------------ the other workloads
MASK_WITH_E4M3 = 0b11011


def _timed(fn):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def cfg1_fp64(E, ctx) -> dict:
    """L=32, n=1024, nb=128, beta=4: plain FP64 tile Cholesky + 64 samples (seed 0)."""
    import torch

    L, nb, beta, s = 32, 128, 4.0, 64
    n = L * L
    ms = []
    for it in range(6):
        A = E.emu_cov_build(ctx, L, beta, nb)
        info = E.emu_potrf_mp(ctx, A)
        if it > 0:
            ms.append(info.ms)
        if it < 5:
            A.free()
    Y, ts = _timed(lambda: E.emu_sample(ctx, A, s, seed=0))
    Lf = E.emu_mat_export(ctx, A)
    A.free()
    S = E.emu_cov_build(ctx, L, beta, nb)
    Sd = E.emu_mat_export(ctx, S)
    S.free()
    Sd = Sd + Sd.t() - torch.diag(torch.diag(Sd))
    be = float(torch.linalg.norm(Lf @ Lf.t() - Sd) / torch.linalg.norm(Sd))
    fm = statistics.median(ms)
    return {"workload": "L=32 n=1024 nb=128 beta=4, plain FP64 tile Cholesky + 64 samples seed 0",
            "factor_ms": round(fm, 4), "tflops": round(n ** 3 / 3 / (fm * 1e-3) / 1e12, 4),
            "sample_ms": round(ts * 1e3, 3), "backward_error": be,
            "parity": "vs the CPU oracle to 1e-12 in tests/test_gpu_fp64.py"}


def cfg3_e4m3_refine(E, ctx) -> dict:
    """L=256, n=65536, nb=1024, beta=12: adaptive FP64/FP32/BF16/E4M3 at eps=1e-6, 16 N(0,1) right-hand sides
    refined with FP64 residuals; the all-FP64-class tensor-core factor of the same matrix beside it."""
    import torch

    L, nb, beta, eps = 256, 1024, 12.0, 1e-6
    n = L * L
    flops = n ** 3 / 3
    S = E.emu_cov_build(ctx, L, beta, nb)
    ms, info = [], None
    for it in range(5):  # the first four factors of a signature try the tuner's choices
        A = E.emu_mat_clone(ctx, S)
        info = E.emu_potrf_mp(ctx, A, eps=eps, prec_mask=MASK_WITH_E4M3)
        ms.append(info.ms)
        if it < 4:
            A.free()
    g = torch.Generator(device="cpu").manual_seed(4)
    B = torch.randn((16, n), generator=g, dtype=torch.float64).cuda().t()  # n x 16, column-major
    E.emu_solve_refine(ctx, A, S, B, tol=1e-12, maxit=30)  # warm-up
    (X, ri), _ = _timed(lambda: E.emu_solve_refine(ctx, A, S, B, tol=1e-12, maxit=30))
    est = E.emu_backward_error_est(ctx, A, L, beta, nprobes=8, seed=5)
    A.free()
    out = {"workload": "L=256 n=65536 nb=1024 beta=12, adaptive FP64/FP32/BF16/E4M3 at eps=1e-6; 16 N(0,1) "
                       "right-hand sides, FP64-residual refinement to 1e-12",
           "tiles_per_class": dict(zip(E.CLASS_NAMES, info.tiles)), "factor_ms": round(ms[-1], 2),
           "factor_ms_tuning": [round(x, 2) for x in ms[:4]], "tflops": round(flops / (ms[-1] * 1e-3) / 1e12, 2),
           "backward_error_est": est, "refine_iters": ri.iters, "refine_ms": round(ri.ms, 2),
           "refine_backward_error": ri.rel_resid}
    A = E.emu_mat_clone(ctx, S)
    S.free()
    i64 = E.emu_potrf_mp(ctx, A, eps=eps, prec_mask=1)
    out["fp64_class_tc_factor_ms"] = round(i64.ms, 2)
    out["fp64_class_tc_tflops"] = round(flops / (i64.ms * 1e-3) / 1e12, 3)
    out["fp64_class_tc_backward_error_est"] = E.emu_backward_error_est(ctx, A, L, beta, nprobes=8, seed=5)
    out["speedup_vs_fp64_class_tc"] = round(i64.ms / ms[-1], 2)
    A.free()
    out["fp64_pipe"] = ("not run in the default bench (about 80 s at the DFMA rate); see --workload fp64_L400 "
                        "for the plain FP64 factor at scale")
    return out


def cfg4_classfmt(E, ctx, samples: int = 1024) -> dict:
    """L=480, n=230400, nb=1024, beta=16: BF16/E4M3-dominant class-format storage at eps=1e-6, 1024 samples
    (seed 2), backward error by the Hutchinson estimate (S regenerated from its parameters)."""
    import torch

    L, nb, beta, eps = 480, 1024, 16.0, 1e-6
    n = L * L
    flops = n ** 3 / 3
    A, tb = _timed(lambda: E.emu_cov_build_classfmt(ctx, L, beta, nb, eps=eps, prec_mask=MASK_WITH_E4M3))
    free0, _ = torch.cuda.mem_get_info()
    info = E.emu_potrf_mp(ctx, A, eps=eps)
    Y = E._colmajor_empty(n, samples, ctx.device)
    _, ts = _timed(lambda: E.emu_sample(ctx, A, samples, seed=2, out=Y))
    est, te = _timed(lambda: E.emu_backward_error_est(ctx, A, L, beta, nprobes=8, seed=5))
    sizes = {"fp64": 8, "fp32": 4, "tf32": 4, "bf16": 2, "e4m3": 1}
    stored = sum(c * nb * nb * sizes[k] for k, c in zip(E.CLASS_NAMES, info.tiles))
    A.free()
    del Y
    return {"workload": "L=480 n=230400 nb=1024 beta=16, class-format storage at eps=1e-6 (every tile in its "
                        "class's format), 1024 samples seed 2",
            "tiles_per_class": dict(zip(E.CLASS_NAMES, info.tiles)), "stored_gb": round(stored / 1e9, 2),
            "fp64_lower_gb": round((n // nb + 1) * (n // nb + 2) / 2 * nb * nb * 8 / 1e9, 1),
            "build_s": round(tb, 3), "factor_ms": round(info.ms, 1),
            "tflops": round(flops / (info.ms * 1e-3) / 1e12, 2), "sample_ms": round(ts * 1e3, 1),
            "backward_error_est": est, "estimate_probes": 8, "estimate_s": round(te, 2),
            "device_free_gb_after_build": round(free0 / 1e9, 1)}


def cfg5_batched(E, ctx, seed: int = 3, count: int = 1024, s: int = 256) -> dict:
    """1024 covariances, L ~ U{8..64}, beta ~ U[2,8) (SplitMix64 draws, seed 3), eps=1e-8, 256 samples each,
    one call in one captured graph with the tuned tile size; plain FP64 batch and per-matrix FP64 beside it."""
    import torch

    from paper_2408_04440_gb300.inputs import batch_draws

    draws = batch_draws(count, seed)
    flops = sum((L * L) ** 3 / 3.0 for L, _ in draws)
    Ys = [E._colmajor_empty(L * L, s, ctx.device) for L, _ in draws]

    def step(nb=0, e=1e-8):
        return E.emu_batch_potrf_sample(ctx, draws, nb=nb, eps=e, prec_mask=MASK_FP64_FP32_BF16, nsamples=s,
                                        seed=seed, out_Y=Ys)

    _, _, infos, _ = step()  # tunes the tile size, captures the graph
    ms = []
    for _ in range(3):
        _, _, infos, _ = step()
        ms.append(infos[0].ms)
    nb_used = infos[0].nb
    m = statistics.median(ms)
    step(nb=nb_used, e=0.0)
    _, _, i64, _ = step(nb=nb_used, e=0.0)
    E.emu_batch_release(ctx)
    sub = draws[:128]
    fl_sub = sum((L * L) ** 3 / 3.0 for L, _ in sub)

    def per_matrix():
        for b, (L, beta) in enumerate(sub):
            M = E.emu_cov_build(ctx, L, beta, 256)
            E.emu_potrf_mp(ctx, M)
            E.emu_sample(ctx, M, s, seed=seed, stream_id=b)
            M.free()

    per_matrix()
    _, dt = _timed(per_matrix)
    del Ys
    return {"workload": "1024 covariances L~U{8..64} beta~U[2,8) seed 3, eps=1e-8, 256 samples each, one call",
            "call_ms": round(m, 2), "tflops": round(flops / (m * 1e-3) / 1e12, 3), "tile_size": nb_used,
            "fp64_batch_ms": round(i64[0].ms, 2), "per_matrix_fp64_tflops": round(fl_sub / dt / 1e12, 4),
            "speedup_vs_per_matrix_fp64": round(flops / (m * 1e-3) / (fl_sub / dt), 2)}


def fp64tc_headline(E, ctx, a, flops, mixed_ms) -> dict:
    """The headline matrix with every tile FP64-class (exact digit products on the BF16 tensor cores)."""
    ms = []
    for it in range(2):
        A = E.emu_cov_build(ctx, a.L, a.beta, a.nb)
        info = E.emu_potrf_mp(ctx, A, eps=a.eps, prec_mask=1)
        ms.append(info.ms)
        if it == 1:
            est = E.emu_backward_error_est(ctx, A, a.L, a.beta, nprobes=8, seed=5)
        A.free()
    return {"factor_ms": round(ms[-1], 3), "tflops": round(flops / (ms[-1] * 1e-3) / 1e12, 3),
            "backward_error_est": est, "speedup_of_mixed": round(ms[-1] / mixed_ms, 2),
            "note": "FP64-accurate factor on the tensor cores (Ozaki digits); the plain FP64 row is the FP64 pipe"}


def other_configs(E, ctx, a, flops, mixed_ms) -> dict:
    import torch

    out = {}
    todo = [c for c in a.configs.split(",") if c]
    fns = {"cfg1": lambda: cfg1_fp64(E, ctx), "fp64tc": lambda: fp64tc_headline(E, ctx, a, flops, mixed_ms),
           "cfg3": lambda: cfg3_e4m3_refine(E, ctx), "cfg5": lambda: cfg5_batched(E, ctx),
           "cfg4": lambda: cfg4_classfmt(E, ctx)}
    for c in ["cfg1", "fp64tc", "cfg3", "cfg5", "cfg4"]:
        if c not in todo:
            continue
        t0 = time.perf_counter()
        try:
            out[c] = fns[c]()
        except Exception as exc:  # one workload's failure is reported, not fatal to the line
            out[c] = {"error": f"{type(exc).__name__}: {exc}"}
        out[c]["wall_s"] = round(time.perf_counter() - t0, 2)
        torch.cuda.empty_cache()
    return out


def _panel_flops(n: int, nb: int, k: int) -> float:
    m = max(n - (k + 1) * nb, 0)
    kb = min(nb, n - k * nb)
    return kb ** 3 / 3.0 + m * kb * kb + m * m * kb


def cpu_baseline(a, budget_s: float = 15.0) -> dict:
    """The oracle, as it stands, on this host's cores: the first panel steps of
    the same n=16384 blocked factor (as many as fit in about budget_s)."""
    import oracle as O

    n, nb = a.L * a.L, a.nb
    S = O.cov_build(a.L, a.beta)
    NT = (n + nb - 1) // nb
    fl, dt, k = 0.0, 0.0, 0
    while k < NT and dt < budget_s:
        t0 = time.perf_counter()
        O.lib().orc_potrf_blocked_steps(n, nb, O._dp(S), n, k, k + 1)
        dt += time.perf_counter() - t0
        fl += _panel_flops(n, nb, k)
        k += 1
    return {"value": round(fl / dt / 1e12, 5), "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {k} of {NT} panel steps of the n={n}, nb={nb} FP64 blocked Cholesky "
                      f"({fl:.3e} flop in {dt:.1f} s)"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O

    n, nb = a.L * a.L, a.nb
    NT = (n + nb - 1) // nb
    S = O.cov_build(a.L, a.beta)
    state = {"k": 0}

    def step():
        if state["k"] >= NT:
            S[:, :] = O.cov_build(a.L, a.beta)
            state["k"] = 0
        k = state["k"]
        O.lib().orc_potrf_blocked_steps(n, nb, O._dp(S), n, k, k + 1)
        state["k"] += 1
        return _panel_flops(n, nb, k)

    for _ in range(a.warmup):
        step()
    fl = 0.0
    t0 = time.perf_counter()
    for _ in range(a.steps):
        fl += step()
    dt = time.perf_counter() - t0
    value = fl / dt / 1e12
    cpu = {"value": round(value, 5), "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{a.steps} panel steps of the n={n}, nb={nb} FP64 blocked Cholesky per timed region"}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "TFLOP/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt / max(a.steps, 1) * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "L": a.L, "n": n, "nb": nb},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 5), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- batched
def batched_name(a) -> str:
    return (f"batched: {a.count} covariances, L ~ U{{8..64}} (n = 64..4096), beta ~ U[2,8) (SplitMix64 seed "
            f"{a.batch_seed}), adaptive FP64/FP32/BF16 at eps={a.eps:g}, {a.samples} samples each, one graph")


def run_batched(a):
    import numpy as np
    import torch

    import paper_2408_04440_gb300 as E
    from paper_2408_04440_gb300 import build as _b
    from paper_2408_04440_gb300.inputs import batch_draws

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if rank == 0 or world == 1:
        _b.build()
    if dist is not None:
        dist.barrier()
    eps = a.eps
    s = a.samples
    draws = batch_draws(a.count, a.batch_seed + rank)  # weak scaling: a batch per rank
    flops = sum((L * L) ** 3 / 3.0 for L, _ in draws)
    stream = torch.cuda.Stream()
    ctx = E.Context(local, stream=stream)
    Ys = [E._colmajor_empty(L * L, s, ctx.device) for L, _ in draws]

    def step(nb=0, e=eps):
        return E.emu_batch_potrf_sample(ctx, draws, nb=nb, eps=e, prec_mask=MASK_FP64_FP32_BF16, nsamples=s,
                                        seed=a.seed, out_Y=Ys)

    with torch.cuda.stream(stream):
        for _ in range(max(a.warmup, 1)):  # the first call tunes the tile size and captures the graph
            _, _, infos, _ = step()
        clocks = ClockSampler(local)
        barrier()
        launches0 = ctx.launch_count
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            step()
        e1.record(stream)
        stream.synchronize()
        barrier()
        clk = clocks.stop()
        gpu_launches = ctx.launch_count - launches0
        t = torch.tensor([e0.elapsed_time(e1)], device=ctx.device)
        if dist is not None:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item()) / a.steps
        value = world * flops / (ms_per_step * 1e-3) / 1e12
        if rank != 0:
            ctx.close()
            if dist is not None:
                dist.barrier()
                dist.destroy_process_group()
            return
        nb_used = infos[0].nb
        tiles = [int(x) for x in np.sum([i.tiles for i in infos], axis=0)]
        extra = {"tile_size": nb_used, "tiles_per_class": dict(zip(E.CLASS_NAMES, tiles)), "graph_ms": round(infos[0].ms, 3)}
        ctx.prof_enable(True)
        step()
        prof = ctx.prof_read()
        ctx.prof_enable(False)
        step_ms = sum(v["ms"] for v in prof.values())
        extra["kernel_groups"] = {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                      "share": round(v["ms"] / step_ms, 4)} for k, v in prof.items() if v["launches"]}
        roof = roofline(prof, load_peaks())
        # the comparisons: the whole batch in plain FP64, and the single-matrix
        # FP64 path launched matrix by matrix (a sample, scaled by its flops)
        if not a.no_fp64:
            step(nb=nb_used, e=0.0)
            _, _, i64, _ = step(nb=nb_used, e=0.0)
            E.emu_batch_release(ctx)
            extra["fp64_batch_ms"] = round(i64[0].ms, 2)
            extra["fp64_batch_tflops"] = round(flops / (i64[0].ms * 1e-3) / 1e12, 4)
            sub = draws[:128]
            fl_sub = sum((L * L) ** 3 / 3.0 for L, _ in sub)

            def per_matrix():
                for b, (L, beta) in enumerate(sub):
                    M = E.emu_cov_build(ctx, L, beta, 256)
                    E.emu_potrf_mp(ctx, M)
                    E.emu_sample(ctx, M, s, seed=a.seed, stream_id=b)
                    M.free()

            per_matrix()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            per_matrix()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            extra["per_matrix_fp64_tflops"] = round(fl_sub / dt / 1e12, 4)
            extra["per_matrix_fp64_sample"] = "first 128 matrices, single-matrix FP64 path, one call each"
            extra["speedup_vs_per_matrix_fp64"] = round(value / (fl_sub / dt / 1e12), 2)
        e2e = None
        if not a.no_e2e:
            # the same call with every Y_b read back into pinned host memory
            hY = [torch.empty((s, L * L), dtype=torch.float64, pin_memory=True).t() for L, _ in draws]
            step()
            for h, y in zip(hY, Ys):
                h.copy_(y, non_blocking=True)
            torch.cuda.synchronize()
            k = max(3, min(a.steps, 5))
            t0 = time.perf_counter()
            for _ in range(k):
                step()
                for h, y in zip(hY, Ys):
                    h.copy_(y, non_blocking=True)
                torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / k
            e2e = {"value": round(flops / dt / 1e12, 4), "unit": "TFLOP/s", "ms_per_step": round(dt * 1e3, 3),
                   "h2d_bytes_per_step": a.count * 32, "d2h_bytes_per_step": int(sum(L * L * s * 8 for L, _ in draws)),
                   "steps": k, "path": "emu_batch_potrf_sample (parameters in, samples to pinned host memory)"}
    cpu = None if (a.no_cpu or world > 1) else cpu_baseline_batched(a, draws)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed:f64+f32(3xbf16 split)+bf16", "data": "synthetic",
        "config": {"workload": batched_name(a), "count": a.count, "eps": eps, "samples": s, "seed": a.seed,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2: every step rebuilds the ~19 GB FP64 tile arena"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clk,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def _oracle_matrix_flops(L, beta, s, seed, b):
    """One matrix of the batch through the oracle: build, blocked FP64 factor
    (tile 256), samples; returns the factor's n^3/3."""
    import oracle as O

    n = L * L
    S = O.cov_build(L, beta)
    Lf, _ = O.potrf_blocked(S, 256)
    O.trmm_lower(Lf, O.normal_matrix(seed, b, n, s))
    return n ** 3 / 3.0


def cpu_baseline_batched(a, draws, budget_s: float = 15.0) -> dict:
    """The oracle on this host's cores, matrix after matrix of the batch until
    about budget_s has passed."""
    fl, dt, m = 0.0, 0.0, 0
    while m < len(draws) and dt < budget_s:
        t0 = time.perf_counter()
        fl += _oracle_matrix_flops(draws[m][0], draws[m][1], a.samples, a.seed, m)
        dt += time.perf_counter() - t0
        m += 1
    return {"value": round(fl / dt / 1e12, 5), "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {m} of {len(draws)} matrices: build, blocked FP64 factor, {a.samples} samples "
                      f"({fl:.3e} flop in {dt:.1f} s)"}


def run_reference_batched(a):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from paper_2408_04440_gb300.inputs import batch_draws

    draws = batch_draws(a.count, a.batch_seed)
    state = {"m": 0}

    def step():
        m = state["m"] % len(draws)
        state["m"] += 1
        return _oracle_matrix_flops(draws[m][0], draws[m][1], a.samples, a.seed, m)

    for _ in range(a.warmup):
        step()
    fl = 0.0
    t0 = time.perf_counter()
    for _ in range(a.steps):
        fl += step()
    dt = time.perf_counter() - t0
    value = fl / dt / 1e12
    cpu = {"value": round(value, 5), "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{a.steps} matrices of the batch per timed region (one matrix per step)"}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "TFLOP/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt / max(a.steps, 1) * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": batched_name(a), "count": a.count},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 5), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_fp64_L400(a):
    """The FP64 comparison at L=400 (n=160000, nb=1024, beta=16): the plain FP64 tile Cholesky on the FP64 pipe
    (about 104 GB of FP64 lower tiles) and the same factor with every tile FP64-class on the tensor cores in
    class-format storage, each once, with the SM clocks sampled meanwhile."""
    import torch

    import paper_2408_04440_gb300 as E
    from paper_2408_04440_gb300 import build as _b

    _b.build()
    L, nb, beta = 400, 1024, 16.0
    n = L * L
    flops = n ** 3 / 3
    stream = torch.cuda.Stream()
    ctx = E.Context(0, stream=stream)
    out = {"workload": "L=400 n=160000 nb=1024 beta=16: FP64 tile Cholesky", "n": n}
    with torch.cuda.stream(stream):
        W = E.emu_cov_build(ctx, 64, beta, nb)  # warm-up of the FP64 path
        E.emu_potrf_mp(ctx, W)
        W.free()
        clocks = ClockSampler(0)
        A = E.emu_cov_build(ctx, L, beta, nb)
        clocks.start()
        info = E.emu_potrf_mp(ctx, A)
        out["fp64_pipe"] = {"factor_s": round(info.ms / 1e3, 2), "tflops": round(flops / (info.ms * 1e-3) / 1e12, 4),
                            "backward_error_est": E.emu_backward_error_est(ctx, A, L, beta, nprobes=4, seed=5),
                            "clocks": clocks.stop()}
        A.free()
        torch.cuda.empty_cache()
        clocks = ClockSampler(0)
        B = E.emu_cov_build_classfmt(ctx, L, beta, nb, eps=0.0)
        clocks.start()
        info = E.emu_potrf_mp(ctx, B, eps=0.0)
        out["fp64_class_tc"] = {"factor_s": round(info.ms / 1e3, 2),
                                "tflops": round(flops / (info.ms * 1e-3) / 1e12, 3),
                                "backward_error_est": E.emu_backward_error_est(ctx, B, L, beta, nprobes=4, seed=5),
                                "clocks": clocks.stop()}
        B.free()
    print(json.dumps(out), flush=True)
    ctx.close()


def main():
    a = parse()
    if a.workload == "fp64_L400":
        run_fp64_L400(a)
        return
    if a.seed is None:
        a.seed = 3 if a.workload == "batched" else 1
    if a.workload == "batched":
        # the batched workload's own defaults (eps 1e-8, 256 samples, seed 3)
        if a.impl == "reference":
            run_reference_batched(a)
        else:
            run_batched(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
