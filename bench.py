"""Benchmark: formal-solution throughput of FAS V-cycles on one GB300.

Workload: the two-level atom (CRD, 9 Doppler frequencies, A4 rays) in a
64x64x128-cell box (129 nodes in z), eps = 1e-4, exponentially stratified
line-centre optical depth 1e-4..1e4 with seeded log-normal perturbations
(sigma 0.3, k^-5/3 spectrum); 3-grid FAS V-cycles with
(nu0, nu1, nu2, nu3) = (0, 2, 2, 32), FP64 throughout.

One step is one V-cycle, which runs every part of the hot path: formal
solutions on all grids (plane sweeps), MALI rate updates, residuals,
full-weighting restriction, the tau-corrected right-hand side, coarse-grid
iterations, the interpolated relative correction and the convergence check.
value = (nodes x rays x frequencies swept by all formal solutions of the
timed steps) / (summed device time of the steps), in G units/s.

Under torchrun each rank solves its own independently seeded atmosphere
(replicas; no collective touches the solve), and the slowest rank's time
counts.  --impl reference times the FP64 CPU oracle on the host instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "two-level atom, 64x64x129 nodes, eps=1e-4, lognormal sigma=0.3, 3-grid FAS"
GRID = (64, 64, 129)
NU = dict(nu_fmg=16, nu0=0, nu1=2, nu2=2, nu3=32)
N_GRIDS = 3
METRIC = "FS Gvoxel*ray*freq/s (3-grid FAS V-cycle step)"
UNIT = "Gunit/s"
FS_UNITS_PER_FINE = GRID[0] * GRID[1] * GRID[2] * 24 * 9
# FP64 floating-point operations per (node, ray, frequency) of the sweep
# (bilinear I_up 7, new I 5, two accumulations 4, plus 16 per node and ray
# shared by the 9 frequencies for the chi/S interpolation and dtau), and the
# short-characteristics weights (optical path 1, exp 1, u 2, w0 1, w_up 1)
# once per distinct profile value: phi(x) = phi(-x) gives mirror frequencies
# the same optical depth, so 5 of the 9 need their own.  exp and the
# division count as one operation each.
N_DISTINCT_PHI = (9 + 1) // 2
ALG_FLOPS_PER_UNIT = 7 + 5 + 4 + (1 + 1 + 2 + 1 + 1) * N_DISTINCT_PHI / 9.0 + 16.0 / 9.0
FP64_NOMINAL_TFLOPS = 1.25      # GB300, at the 2070 MHz maximum SM clock
# FP32 instructions per unit the FP32 sweep needs (each an FMA-pipe
# instruction): per frequency the bilinear I_up 4, the new I 2 (one of them
# the w_up S_up term shared by a mirror pair is counted per distinct phi
# below), the Jeff sum 1; per distinct phi (5 of 9) the optical path 1, the
# exp2 argument 1, u 1, w0 1, w_up 1, w_up S_up 1, the U sum 1; per node and
# ray the chi0/S bilinear 8 and dtau 2.  Plus per distinct phi one ex2 and one
# rcp on the multi-function unit.
ALG_FP32_OPS_PER_UNIT = 4 + 2 + 1 + 7 * N_DISTINCT_PHI / 9.0 + 10.0 / 9.0
MUFU_EX2_PER_UNIT = MUFU_RCP_PER_UNIT = N_DISTINCT_PHI / 9.0
# DRAM bytes (read + write) of one finest-grid FP64 sweep launch on the bench
# atmosphere per launch shape (ng, bands, threads, lean, stage), from ncu
# captures of the current kernel; a shape the autotuner picks that is not
# listed reports traffic null
FINE_SWEEP_TRAFFIC = {(9, 5, 224, 0, 2): 14835968 + 141922048,
                      (9, 5, 256, 0, 2): 14634752 + 141857536,
                      (9, 5, 448, 0, 2): 13970944 + 144993536,
                      (9, 5, 512, 0, 2): 13957888 + 143129856}
SM_MAX_MHZ = 2070.0


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def replica_seed(rank: int) -> int:
    """Seed of the atmosphere a rank solves: independent replicas, one per rank."""
    return 1 + rank


def aggregate_over_ranks(total_ms: float, units: float, dist=None, device=None):
    """Whole-job figures of a replicated run: the slowest rank's time and the
    units all ranks processed.  ``dist`` is torch.distributed (or None for a
    single process); tensors live on ``device`` (cuda under NCCL, cpu under
    gloo)."""
    if dist is None:
        return total_ms, units
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def build_problem(seed):
    from paper_1701_01607_gb300 import synth
    return synth.stratified_two_level(GRID[0], GRID[1], GRID[2], eps=1e-4, sigma=0.3,
                                      seed=seed)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch

    from paper_1701_01607_gb300 import mg3d as m

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    m.load(build_if_missing=True)
    atm, atom = build_problem(seed=replica_seed(rank))
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    tuning = {}

    fixed = json.loads(args.shapes) if args.shapes else None

    def make(prec):
        h = m.mg3d_create(atm, atom, n_grids=N_GRIDS, fs_prec=prec, **NU)
        m.mg3d_set_stream(h, stream.cuda_stream)
        key = "f64" if prec == m.MG3D_PREC_F64 else "f32"
        if fixed is not None:
            for k, shape in fixed[key].items():
                m.mg3d_set_fs_config(h, int(k), *shape)
            tuning[key] = {"fixed": True,
                           "shapes": {k: m.mg3d_get_fs_config(h, k) for k in range(1, N_GRIDS + 1)}}
        elif not args.no_autotune:
            info = m.mg3d_autotune(h)
            tuning["f64" if prec == m.MG3D_PREC_F64 else "f32"] = {
                "seconds": round(info["seconds"], 3), "candidates": info["evaluated"],
                "shapes": {k: m.mg3d_get_fs_config(h, k) for k in range(1, N_GRIDS + 1)}}
        return h

    def timed_cycles(h, steps, warmup, timing):
        for i in range(warmup):
            m.mg3d_fas_vcycle(h, i == 0)
        m.mg3d_set_timing(h, timing)
        m.mg3d_reset_counters(h)
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.mg3d_fas_vcycle(h, False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, m.mg3d_get_counters(h)

    # ---- measured peak rates of the ALU pipes the sweeps run on (roofline
    # denominators): FP32 FMA, ex2, rcp, FP64 FMA, thread operations per second
    peaks = m.mg3d_probe_alu_peaks(5)
    torch.cuda.synchronize()

    # ---- main measurement: FP64 V-cycles, no per-launch instrumentation
    h = make(m.MG3D_PREC_F64)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ms, cnt = timed_cycles(h, args.steps, args.warmup, timing=False)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms, units = aggregate_over_ranks(sum(ms), cnt["fs_units"], dist, "cuda")
    value = units / (total_ms * 1e-3) / 1e9
    fine = N_GRIDS
    # per-launch sweep times from a separate instrumented pass (event pairs
    # recorded around every sweep inside the replayed V-cycle graph)
    _, cnt_t = timed_cycles(h, max(3, args.steps // 2), 1, timing=True)
    fine_ms = cnt_t["level_fs_kernel_ms"][fine] / max(1, cnt_t["level_fs_timed_launches"][fine])
    fine_units = cnt_t["level_fs_units"][fine] / max(1, cnt_t["level_fs_launches"][fine])

    # ---- end to end: host populations in, V-cycle, host populations out
    nx, ny, nz = GRID
    pinned_in = torch.empty((2, nz, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    pinned_out = torch.empty((2, nz, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    pinned_in[...] = m.mg3d_get_populations(h, fine)
    m.mg3d_set_timing(h, False)
    m.mg3d_reset_counters(h)
    e2e_ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.mg3d_set_populations(h, fine, pinned_in)
        m.mg3d_fas_vcycle(h, False)
        m.mg3d_get_populations(h, fine, pinned_out)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_units = m.mg3d_get_counters(h)["fs_units"]
    launches = cnt["kernel_launches"]
    m.mg3d_destroy(h)

    # ---- mixed precision (FP32 formal solution, FP64 rates): same step
    h32 = make(m.MG3D_PREC_F32)
    ms32, cnt32 = timed_cycles(h32, args.steps, args.warmup, timing=False)
    _, cnt32_t = timed_cycles(h32, max(3, args.steps // 2), 1, timing=True)
    m.mg3d_destroy(h32)
    fine_ms32 = (cnt32_t["level_fs_kernel_ms"][fine]
                 / max(1, cnt32_t["level_fs_timed_launches"][fine]))
    large32 = fp32_sweep_large(m, stream, peaks) if world == 1 and not args.no_large else None

    result = None
    if rank == 0:
        peak = 2.0 * peaks["dfma"] / 1e12       # measured FP64 TFLOP/s
        achieved = ALG_FLOPS_PER_UNIT * fine_units / (fine_ms * 1e-3) / 1e12
        fine_shape = list(tuning.get("f64", {}).get("shapes", {}).get(fine, ()))
        traffic = FINE_SWEEP_TRAFFIC.get(tuple(fine_shape))
        result = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(GRID), "n_grids": N_GRIDS,
                       "n_freq": 9, "rays": 24, **NU, "fs_precision": "f64",
                       "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between timed steps",
                       "sweep_autotune": tuning},
            "roofline": {"kernel": "plane_sweep_kernel<double> (finest grid)", "bound": "alu",
                         "achieved": round(achieved, 4), "peak": round(peak, 4),
                         "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic,
                         "peak_source": "measured FP64 FMA rate x 2 (mg3d_probe_alu_peaks, "
                                        "this run); nominal 1.25 TFLOP/s",
                         "frac_of_nominal": round(achieved / FP64_NOMINAL_TFLOPS, 4),
                         "alg_flops_per_unit": round(ALG_FLOPS_PER_UNIT, 3),
                         "units_per_launch": fine_units,
                         "ms_per_launch": round(fine_ms, 4),
                         "timing": "sweep launches timed in a separate instrumented pass"},
            "roofline_fp32": roofline_fp32(fine_units, fine_ms32, peaks,
                                           "plane_sweep_kernel<float> (finest grid)"),
            "fp32_large_plane": large32,
            "alu_peaks": {"ffma_tops": round(peaks["ffma"] / 1e12, 3),
                          "ex2_tops": round(peaks["ex2"] / 1e12, 3),
                          "rcp_tops": round(peaks["rcp"] / 1e12, 3),
                          "dfma_tops": round(peaks["dfma"] / 1e12, 4),
                          "how": "mg3d_probe_alu_peaks: 8 independent chains per thread, "
                                 "8 blocks of 256 per SM, best of 5 launches"},
            "e2e": {"value": round(e2e_units / (sum(e2e_ms) * 1e-3) / 1e9, 4), "unit": UNIT,
                    "h2d_bytes_per_step": int(pinned_in.nbytes),
                    "d2h_bytes_per_step": int(pinned_out.nbytes)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "mixed_precision": {
                "fs_precision": "f32 (rates f64)",
                "value": round(cnt32["fs_units"] / (sum(ms32) * 1e-3) / 1e9, 4),
                "ms_per_step": round(sum(ms32) / args.steps, 4),
                "fine_sweep_ms": round(fine_ms32, 4),
                "fine_sweep_gunits_s": round(fine_units / (fine_ms32 * 1e-3) / 1e9, 3)},
            "fine_sweep_gunits_s": round(fine_units / (fine_ms * 1e-3) / 1e9, 3),
            "sweep_ms_per_launch_by_level": {
                k: round(cnt["level_fs_kernel_ms"][k] / max(1, cnt["level_fs_timed_launches"][k]), 4)
                for k in range(1, N_GRIDS + 1)},
            "sweep_launches_per_step_by_level": {
                k: cnt["level_fs_launches"][k] // args.steps for k in range(1, N_GRIDS + 1)},
        }
        if not args.no_tts and world == 1:
            result["time_to_solution"] = time_to_solution(m, atm, atom, stream)
            result["mixed_precision"]["accuracy"] = dict(
                result["time_to_solution"]["mixed_precision_fas"],
                what="3-grid FAS from the zero-radiation start to C < 1e-3: FP32 formal "
                     "solution against FP64 throughout; e_inf against a FAS solution "
                     "converged to C < 1e-9")
        if world == 1 and not args.no_cpu:
            result["cpu_baseline"] = cpu_baseline(atm, atom, samples=2)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return result


def roofline_fp32(units, ms, peaks, kernel):
    """FP32 sweep against its ALU roofline: per unit the FP32 instructions of
    the algorithm on the FMA pipes and the ex2/rcp on the multi-function
    unit, at the rates measured in this run; the roofline throughput is the
    slower of the two pipes."""
    t_fma = ALG_FP32_OPS_PER_UNIT / peaks["ffma"]
    t_mufu = MUFU_EX2_PER_UNIT / peaks["ex2"] + MUFU_RCP_PER_UNIT / peaks["rcp"]
    peak = 1.0 / max(t_fma, t_mufu) / 1e9
    achieved = units / (ms * 1e-3) / 1e9
    return {"kernel": kernel, "bound": "alu", "achieved": round(achieved, 3),
            "peak": round(peak, 3), "unit": "Gunit/s", "frac": round(achieved / peak, 4),
            "alg_fp32_ops_per_unit": round(ALG_FP32_OPS_PER_UNIT, 3),
            "mufu_per_unit": round(MUFU_EX2_PER_UNIT + MUFU_RCP_PER_UNIT, 3),
            "limiting_pipe": "fma" if t_fma >= t_mufu else "mufu",
            "units_per_launch": units, "ms_per_launch": round(ms, 4),
            "peak_source": "measured FFMA, ex2 and rcp rates (mg3d_probe_alu_peaks, this run)"}


LARGE_PLANE = (128, 128, 129)


def fp32_sweep_large(m, stream, peaks, reps=10):
    """The FP32 sweep on 128x128 planes (the bench atmosphere's recipe, 129
    nodes in z): 4 times the work per plane step of the 64x64 box, so the
    per-plane barrier and latency weigh less; autotuned, then the sweep
    kernel of `reps` formal solutions timed with CUDA events."""
    from paper_1701_01607_gb300 import synth
    nx, ny, nz = LARGE_PLANE
    atm, atom = synth.stratified_two_level(nx, ny, nz, eps=1e-4, sigma=0.3, seed=1)
    h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32)
    try:
        m.mg3d_set_stream(h, stream.cuda_stream)
        m.mg3d_autotune(h, 1)
        m.mg3d_formal_solve(h, 1, want=False)
        m.mg3d_set_timing(h, True)
        m.mg3d_reset_counters(h)
        for _ in range(reps):
            m.mg3d_formal_solve(h, 1, want=False)
        c = m.mg3d_get_counters(h)
        ms = c["level_fs_kernel_ms"][1] / max(1, c["level_fs_timed_launches"][1])
        shape = m.mg3d_get_fs_config(h, 1)
    finally:
        m.mg3d_destroy(h)
    out = roofline_fp32(nx * ny * nz * 24 * 9, ms, peaks,
                        "plane_sweep_kernel<float>, %dx%dx%d" % LARGE_PLANE)
    out["shape"] = list(shape)
    out["note"] = "sweep kernel alone (events around each launch); not part of the V-cycle step"
    return out


def time_to_solution(m, atm, atom, stream, tol=1e-3):
    """MALI, FAS and FMG from the zero-radiation start to C < tol (FP64), with
    their true error E_inf against a FAS solution converged to C < 1e-9."""
    out = {}
    ref_h = m.mg3d_create(atm, atom, n_grids=N_GRIDS, fs_prec=m.MG3D_PREC_F64, **NU)
    m.mg3d_set_stream(ref_h, stream.cuda_stream)
    m.mg3d_fas_solve(ref_h, 1e-9, 400, n_grids=N_GRIDS)
    n_ref = m.mg3d_get_populations(ref_h, N_GRIDS)
    m.mg3d_destroy(ref_h)
    for method, fn, grids, cap in (("mali", m.mg3d_mali_solve, 1, 200000),
                                   ("fas", m.mg3d_fas_solve, N_GRIDS, 400),
                                   ("fmg", m.mg3d_fmg_solve, N_GRIDS, 400)):
        h = m.mg3d_create(atm, atom, n_grids=grids, fs_prec=m.MG3D_PREC_F64, **NU)
        m.mg3d_set_stream(h, stream.cuda_stream)
        st = fn(h, tol, cap, n_grids=grids)
        n = m.mg3d_get_populations(h, grids)
        m.mg3d_destroy(h)
        out[method] = {"seconds": round(st["seconds"], 4), "iterations": st["iterations"],
                       "fine_fs_equivalents": round(st["fine_fs_equivalents"], 3),
                       "e_inf": float(np.max(np.abs(n - n_ref) / np.abs(n_ref))),
                       "negatives": st["negatives"]}
    out["tol"] = tol
    # the FP32 formal solution (FP64 rates, residuals and transfers) to the
    # same stopping point: its error against the FP64 solve of the same
    # schedule and against the converged reference
    n64 = None
    acc = {}
    for prec, key in ((m.MG3D_PREC_F64, "f64"), (m.MG3D_PREC_F32, "f32")):
        h = m.mg3d_create(atm, atom, n_grids=N_GRIDS, fs_prec=prec, **NU)
        m.mg3d_set_stream(h, stream.cuda_stream)
        st = m.mg3d_fas_solve(h, tol, 400, n_grids=N_GRIDS)
        n = m.mg3d_get_populations(h, N_GRIDS)
        m.mg3d_destroy(h)
        acc[key] = {"cycles": st["iterations"], "seconds": round(st["seconds"], 4),
                    "e_inf": float(np.max(np.abs(n - n_ref) / np.abs(n_ref)))}
        if key == "f64":
            n64 = n
        else:
            acc["f32_vs_f64_e_inf"] = float(np.max(np.abs(n - n64) / np.abs(n64)))
    out["mixed_precision_fas"] = acc
    out["speedup_fas"] = round(out["mali"]["seconds"] / out["fas"]["seconds"], 3)
    out["speedup_fmg"] = round(out["mali"]["seconds"] / out["fmg"]["seconds"], 3)
    out["equal_accuracy"] = equal_accuracy(m, atm, atom, stream, n_ref)
    return out


def equal_accuracy(m, atm, atom, stream, n_ref, target=1e-3):
    """MALI, FAS and FMG, each run until its true error E_inf against the
    converged reference is at most `target` (the same accuracy for all three):
    timed iterations only, the E_inf checks between them are not timed.
    MALI is checked every 5 sweeps, FAS and FMG after every V-cycle (FMG's
    first call is its full-multigrid pass with one V-cycle)."""
    def e_inf(h, grids):
        n = m.mg3d_get_populations(h, grids)
        return float(np.max(np.abs(n - n_ref) / np.abs(n_ref)))

    out = {"target_e_inf": target}
    for method in ("mali", "fas", "fmg"):
        grids = 1 if method == "mali" else N_GRIDS
        h = m.mg3d_create(atm, atom, n_grids=grids, fs_prec=m.MG3D_PREC_F64, **NU)
        m.mg3d_set_stream(h, stream.cuda_stream)
        m.mg3d_reset_counters(h)
        secs, its, err = 0.0, 0, 1.0
        try:
            while err > target and its < 20000:
                t0 = time.perf_counter()
                if method == "mali":
                    m.mg3d_mali_sweep(h, 1, 5)
                    its += 5
                elif method == "fas":
                    m.mg3d_fas_vcycle(h, its == 0)
                    its += 1
                elif its == 0:
                    m.mg3d_fmg_solve(h, 1e300, 1, n_grids=grids)
                    its += 1
                else:
                    m.mg3d_fas_vcycle(h, False)
                    its += 1
                secs += time.perf_counter() - t0
                err = e_inf(h, grids)
            units = m.mg3d_get_counters(h)["fs_units"]
        finally:
            m.mg3d_destroy(h)
        out[method] = {"seconds": round(secs, 4), "iterations": its, "e_inf": err,
                       "fine_fs_equivalents": round(units / FS_UNITS_PER_FINE, 3)}
    out["speedup_fas"] = round(out["mali"]["seconds"] / out["fas"]["seconds"], 3)
    out["speedup_fmg"] = round(out["mali"]["seconds"] / out["fmg"]["seconds"], 3)
    return out



def host_cores() -> int:
    """Cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_time_oracle_fs(atm, atom, samples, threads):
    """Seconds for `samples` fine-grid formal solutions of the FP64 oracle
    with `threads` host threads (1: its plain serial loop)."""
    from oracle import mg3d_oracle as O
    prob = O.TwoLevelProblem(atm, atom, n_grids=1)
    prob.threads = threads
    n = prob.zero_radiation(1)
    prob.formal_solution(1, n)          # warm-up (page-in, thread pool)
    t0 = time.perf_counter()
    for _ in range(samples):
        prob.formal_solution(1, n)
    return time.perf_counter() - t0


def cpu_baseline(atm, atom, samples=2):
    """The FP64 CPU oracle as it stands: fine-grid formal solutions (the
    unit of the metric; not V-cycles), on all of the host's cores (rays on
    separate threads) and on one."""
    from oracle import mg3d_oracle as O
    cores = min(host_cores(), O.max_threads()) if O.max_threads() > 1 else 1
    many = max(samples, 4 * min(cores, 24) // 4)
    dt_all = cpu_time_oracle_fs(atm, atom, many, cores)
    dt_one = cpu_time_oracle_fs(atm, atom, samples, 1)
    return {"value": round(many * FS_UNITS_PER_FINE / dt_all / 1e9, 6), "unit": UNIT,
            "cores": cores, "kind": "oracle",
            "sample": f"{many} fine-grid formal solutions of the 64x64x129 box "
                      f"({many * FS_UNITS_PER_FINE:.3g} units, {dt_all:.1f} s) on {cores} "
                      f"threads (rays in parallel); formal solutions only, not V-cycles",
            "single_thread": {"value": round(samples * FS_UNITS_PER_FINE / dt_one / 1e9, 6),
                              "unit": UNIT, "cores": 1,
                              "sample": f"{samples} fine-grid formal solutions, {dt_one:.1f} s"}}


# ---------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return None
    atm, atom = build_problem(seed=1)
    from oracle import mg3d_oracle as O
    cores = min(host_cores(), O.max_threads()) if O.max_threads() > 1 else 1
    prob = O.TwoLevelProblem(atm, atom, n_grids=1)
    prob.threads = cores
    n = prob.zero_radiation(1)
    for _ in range(args.warmup):
        prob.formal_solution(1, n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        prob.formal_solution(1, n)
    dt = time.perf_counter() - t0
    value = args.steps * FS_UNITS_PER_FINE / dt / 1e9
    sample = (f"{args.steps} fine-grid formal solutions of the 64x64x129 box per run, one per "
              f"step, FP64 C oracle on {cores} host threads (rays in parallel); it times "
              f"formal solutions, the metric's unit, not V-cycles")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(GRID), "fs_precision": "f64"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_profile_case(prec_name, launches, shape):
    """A few finest-grid formal solutions of the bench workload, for ncu.

    ``shape`` "ng,bands,threads[,lean[,stage]]" fixes the sweep's launch shape (e.g. the one
    the autotuner chose in a bench run); empty keeps the library default.
    No autotuning runs here, so every sweep launch is a profiled one."""
    from paper_1701_01607_gb300 import mg3d as m
    m.load(build_if_missing=True)
    atm, atom = build_problem(seed=1)
    prec = m.MG3D_PREC_F64 if prec_name == "f64" else m.MG3D_PREC_F32
    h = m.mg3d_create(atm, atom, n_grids=N_GRIDS, fs_prec=prec, **NU)
    try:
        if shape:
            vals = [int(v) for v in shape.split(",")]
            m.mg3d_set_fs_config(h, N_GRIDS, *vals)
        for _ in range(launches):
            m.mg3d_formal_solve(h, N_GRIDS, want=False)
        print("profile case:", prec_name, m.mg3d_get_fs_config(h, N_GRIDS), flush=True)
    finally:
        m.mg3d_destroy(h)


BATCH_SIZES = [(32, 32, 33), (48, 48, 97), (64, 64, 129), (96, 96, 193)]


def batch_members(n=32, seed0=100, ml_chunk=100):
    """The 32-atmosphere batch: seeds seed0 .. seed0+n-1, sizes drawn from
    BATCH_SIZES by each seed, two-level atoms (9 frequencies) for even seeds
    and the 6-level atom (600 frequencies) for odd seeds; FP32 formal
    solution, FP64 rates, 3 grids.  Returns (kind, atmosphere, atom) tuples."""
    from paper_1701_01607_gb300 import synth
    ml_atom = synth.hydrogen_like_atom(line_freq=100, cont_freq=20, seed=2)
    out = []
    for i in range(n):
        seed = seed0 + i
        nx, ny, nz = BATCH_SIZES[int(np.random.default_rng(seed).integers(len(BATCH_SIZES)))]
        if seed % 2 == 0:
            atm, atom = synth.stratified_two_level(nx, ny, nz, eps=1e-3, sigma=0.3, seed=seed)
            out.append(("two", atm, atom))
        else:
            out.append(("ml", synth.chromosphere(nx, ny, nz, ml_atom, seed=seed), ml_atom))
    return out


def run_batch(args):
    """Batched V-cycles of the 32-atmosphere batch (opt-in, --batch): one
    batched sweep launch per atom kind (per frequency chunk for the 6-level
    members), V-cycles replayed from CUDA graphs.  Prints one JSON line."""
    import torch

    from paper_1701_01607_gb300 import mg3d as m
    m.load(build_if_missing=True)
    t0 = time.perf_counter()
    spec = batch_members()
    params = dict(n_grids=3, fs_prec=m.MG3D_PREC_F32, nu_fmg=16, nu0=10, nu1=2, nu2=4,
                  nu3=32)
    hs = []
    for kind, atm, atom in spec:
        if kind == "two":
            hs.append(m.mg3d_create(atm, atom, **params))
        else:
            hs.append(m.mg3d_create_ml(atm, atom, ml_chunk=100, **params))
    b = m.mg3d_batch_create(hs)
    setup_s = time.perf_counter() - t0
    free, total = torch.cuda.mem_get_info()
    try:
        for i in range(args.warmup):
            m.mg3d_batch_fas_vcycle(b, len(hs), i == 0)
        c0 = m.mg3d_batch_counters(b)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            C = m.mg3d_batch_fas_vcycle(b, len(hs), False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t1
        c1 = m.mg3d_batch_counters(b)
    finally:
        m.mg3d_batch_destroy(b)
        for h in hs:
            m.mg3d_destroy(h)
    units = c1["fs_units"] - c0["fs_units"]
    kinds = [k for k, _, _ in spec]
    # the same members alone, one handle at a time, same schedule and steps:
    # the aggregate throughput the batch replaces
    solo_wall, solo_units = 0.0, 0.0
    for kind, atm, atom in spec:
        h = (m.mg3d_create(atm, atom, **params) if kind == "two"
             else m.mg3d_create_ml(atm, atom, ml_chunk=100, **params))
        try:
            for i in range(args.warmup):
                m.mg3d_fas_vcycle(h, i == 0)
            u0 = m.mg3d_get_counters(h)["fs_units"]
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for _ in range(args.steps):
                m.mg3d_fas_vcycle(h, False)
            torch.cuda.synchronize()
            solo_wall += time.perf_counter() - t1
            solo_units += m.mg3d_get_counters(h)["fs_units"] - u0
        finally:
            m.mg3d_destroy(h)
    solo = solo_units / solo_wall / 1e9
    return {"metric": "batched FS Gvoxel*ray*freq/s (32 uneven atmospheres, 3-grid FAS V-cycle)",
            "value": round(units / wall / 1e9, 4), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(wall / args.steps * 1e3, 2), "higher_is_better": True,
            "dtype": "f32 formal solution, f64 rates", "data": "synthetic",
            "config": {"workload": "32 atmospheres, seeds 100-131, sizes from "
                                   + ", ".join("x".join(map(str, s)) for s in BATCH_SIZES),
                       "two_level_members": kinds.count("two"),
                       "six_level_members": kinds.count("ml"),
                       "freq_per_chunk_six_level": 100, **params},
            "gpu_launches_per_step": round((c1["kernel_launches"] - c0["kernel_launches"])
                                           / args.steps, 1),
            "device_gb_in_use": round((total - free) / 1e9, 1), "setup_s": round(setup_s, 1),
            "max_rel_change_last_step": float(np.max(C)),
            "solo": {"value": round(solo, 4), "unit": UNIT,
                     "ms_per_step": round(solo_wall / args.steps * 1e3, 2),
                     "what": "each member alone on its own handle, one after the other, same "
                             "schedule, warm-up and timed V-cycles"},
            "batch_over_solo": round(units / wall / 1e9 / solo, 3)}


def run_scattering(args):
    """Background coherent scattering (Sec. 4.8) against convergence: MALI
    and 3-grid FAS from the zero-radiation start (with its Lambda-iteration)
    until the true error E_inf against a FAS solution converged to C < 1e-9
    is <= 1e-3, for grey scattering opacities of 0, 1, 10 and 100 times the
    thermal continuum opacity.  32x32x65 chromosphere, 6-level atom with 120
    frequencies, collisions out of the ground level weakened 1e3 times (so
    the resonance lines scatter too), FP64 throughout.  Opt-in,
    --scattering-experiment; prints one JSON line."""
    from paper_1701_01607_gb300 import mg3d as m
    from paper_1701_01607_gb300 import synth
    m.load(build_if_missing=True)
    atom = synth.hydrogen_like_atom(line_freq=20, cont_freq=4, seed=2)
    params = dict(fs_prec=m.MG3D_PREC_F64, nu_fmg=16, nu0=20, nu1=4, nu2=8, nu3=32)
    out = {"metric": "iterations and seconds to E_inf <= 1e-3 against background scattering",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "chromosphere 32x32x65, 6-level atom, 120 frequencies, seed 2",
                      "ground_collisions": 1e-3, "target_e_inf": 1e-3, **params}}
    for scat in (0.0, 1.0, 10.0, 100.0):
        atm = synth.chromosphere(32, 32, 65, atom, seed=2, ground_collisions=1e-3,
                                 scattering=scat)
        ref = m.mg3d_create_ml(atm, atom, n_grids=3, **params)
        try:
            m.mg3d_fas_solve(ref, 1e-9, 400, n_grids=3)
            n_ref = m.mg3d_get_populations(ref, 3)
        finally:
            m.mg3d_destroy(ref)
        row = {}
        for method, grids, cap in (("mali", 1, 2000), ("fas", 3, 60)):
            h = m.mg3d_create_ml(atm, atom, n_grids=grids, **params)
            secs, errs, cs = 0.0, [], []
            try:
                m.mg3d_init_zero_radiation(h, grids)
                for it in range(cap):
                    t0 = time.perf_counter()
                    if method == "mali":
                        c = m.mg3d_mali_sweep(h, 1, 1)
                    else:
                        c = m.mg3d_fas_vcycle(h, it == 0)
                    secs += time.perf_counter() - t0
                    n = m.mg3d_get_populations(h, grids)
                    errs.append(float(np.max(np.abs(n - n_ref) / np.abs(n_ref))))
                    cs.append(float(c))
                    if errs[-1] <= 1e-3:
                        break
            finally:
                m.mg3d_destroy(h)
            row[method] = {"reached": errs[-1] <= 1e-3, "iterations": len(errs),
                           "seconds": round(secs, 3), "e_inf_last": float(f"{errs[-1]:.3g}"),
                           "c_last": float(f"{cs[-1]:.3g}"),
                           "c_first": [float(f"{x:.3g}") for x in cs[:6]]}
        out[f"scattering_{scat:g}"] = row
    return out


def _to_target(m, make, grids, n_ref, step, cap, target=1e-3):
    """Iterations (step(h, it)) of a fresh handle until the true error
    E_inf against n_ref is <= target; wall time of the steps only."""
    h = make()
    secs, errs = 0.0, []
    try:
        for it in range(cap):
            t0 = time.perf_counter()
            step(h, it)
            secs += time.perf_counter() - t0
            n = m.mg3d_get_populations(h, grids)
            errs.append(float(np.max(np.abs(n - n_ref) / np.abs(n_ref))))
            if errs[-1] <= target:
                break
    finally:
        m.mg3d_destroy(h)
    return {"reached": errs[-1] <= target, "iterations": len(errs), "seconds": round(secs, 3),
            "e_inf_last": float(f"{errs[-1]:.3g}")}


def run_velocity(args):
    """Moving atmospheres (CRD with Doppler-shifted profiles): the 64x64x129
    box (eps = 1e-4, sigma = 0.3) with a 17-point frequency grid on
    [-5, 5] Doppler widths, static and with a seeded velocity field of rms 1
    Doppler width; FP64 MALI and 3-grid FAS to E_inf <= 1e-3 against each
    case's FAS reference converged to C < 1e-9, and the autotuned sweep time
    of each case in FP64 and FP32.  Opt-in, --velocity-experiment; prints one
    JSON line."""
    from paper_1701_01607_gb300 import mg3d as m
    from paper_1701_01607_gb300 import synth
    m.load(build_if_missing=True)
    atom = synth.TwoLevelAtom(n_freq=17, x_max=5.0)
    out = {"metric": "iterations and seconds to E_inf <= 1e-3; sweep ms per launch",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "64x64x129 two-level box, eps 1e-4, sigma 0.3, seed 1, "
                                  "17 frequencies on [-5, 5]", "nu": NU, "target_e_inf": 1e-3}}
    for vel in (0.0, 1.0):
        atm, _ = synth.stratified_two_level(GRID[0], GRID[1], GRID[2], eps=1e-4, sigma=0.3,
                                            seed=1, atom=atom, velocity=vel)
        ref = m.mg3d_create(atm, atom, n_grids=3, **NU)
        m.mg3d_fas_solve(ref, 1e-9, 400, n_grids=3)
        n_ref = m.mg3d_get_populations(ref, 3)
        m.mg3d_destroy(ref)
        row = {"fas": _to_target(m, lambda: m.mg3d_create(atm, atom, n_grids=3, **NU), 3, n_ref,
                                 lambda h, it: m.mg3d_fas_vcycle(h, it == 0), 60),
               "mali": _to_target(m, lambda: m.mg3d_create(atm, atom, n_grids=1, **NU), 1, n_ref,
                                  lambda h, it: m.mg3d_mali_sweep(h, 1, 1), 3000)}
        for prec, pname in ((m.MG3D_PREC_F64, "f64"), (m.MG3D_PREC_F32, "f32")):
            h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=prec, **NU)
            try:
                m.mg3d_autotune(h)
                m.mg3d_set_timing(h, True)
                m.mg3d_reset_counters(h)
                for _ in range(5):
                    m.mg3d_formal_solve(h, 1, want=False)
                c = m.mg3d_get_counters(h)
                row[f"sweep_{pname}"] = {
                    "ms": round(c["fs_kernel_ms"] / c["fs_timed_launches"], 3),
                    "gunits_s": round(c["fs_units"] / (c["fs_kernel_ms"] * 1e-3) / 1e9, 2),
                    "shape": list(m.mg3d_get_fs_config(h, 1))}
            finally:
                m.mg3d_destroy(h)
        out["moving" if vel else "static"] = row
    # the 6-level atom: sweep cost on the 64x64x129 chromosphere (120
    # frequencies), convergence on a 32x32x65 one with the ground-level
    # collisions weakened 1e3 times (resonance lines scattering)
    ml_atom = synth.hydrogen_like_atom(line_freq=20, cont_freq=4, seed=2)
    ml = {}
    for vel in (0.0, 1.0):
        key = "moving" if vel else "static"
        atm = synth.chromosphere(64, 64, 129, ml_atom, seed=2, velocity=vel)
        for prec, pname in ((m.MG3D_PREC_F32, "f32"), (m.MG3D_PREC_F64, "f64")):
            h = m.mg3d_create_ml(atm, ml_atom, n_grids=1, fs_prec=prec)
            try:
                m.mg3d_autotune(h)
                m.mg3d_set_timing(h, True)
                m.mg3d_reset_counters(h)
                for _ in range(3):
                    m.mg3d_formal_solve_ml(h, 1)
                c = m.mg3d_get_counters(h)
                ml[f"{key}_sweep_{pname}"] = {
                    "ms": round(c["fs_kernel_ms"] / c["fs_timed_launches"], 3),
                    "gunits_s": round(c["fs_units"] / (c["fs_kernel_ms"] * 1e-3) / 1e9, 2),
                    "shape": list(m.mg3d_get_ml_shape(h, 1))}
            finally:
                m.mg3d_destroy(h)
        atm = synth.chromosphere(32, 32, 65, ml_atom, seed=2, ground_collisions=1e-3,
                                 velocity=vel)
        mp = dict(fs_prec=m.MG3D_PREC_F64, nu_fmg=16, nu0=20, nu1=4, nu2=8, nu3=32)
        ref = m.mg3d_create_ml(atm, ml_atom, n_grids=3, **mp)
        m.mg3d_fas_solve(ref, 1e-9, 400, n_grids=3)
        n_ref = m.mg3d_get_populations(ref, 3)
        m.mg3d_destroy(ref)
        ml[f"{key}_fas"] = _to_target(m, lambda: m.mg3d_create_ml(atm, ml_atom, n_grids=3, **mp),
                                      3, n_ref, lambda h, it: m.mg3d_fas_vcycle(h, it == 0), 60)
        ml[f"{key}_mali"] = _to_target(m, lambda: m.mg3d_create_ml(atm, ml_atom, n_grids=1, **mp),
                                       1, n_ref, lambda h, it: m.mg3d_mali_sweep(h, 1, 1), 2000)
    out["six_level"] = ml
    return out


def run_prd(args):
    """Partial redistribution (two-level atom): the 64x64x129 box (eps =
    1e-4, sigma = 0.3) with 17 frequencies on [-5, 5] Doppler widths and
    coherence fractions 0 (CRD), 0.5 and 1; FP64 MALI and 3-grid FAS to
    E_inf <= 1e-3 against each case's FAS reference converged to C < 1e-9,
    and the autotuned sweep time in FP64 and FP32.  Opt-in,
    --prd-experiment; prints one JSON line."""
    from paper_1701_01607_gb300 import mg3d as m
    from paper_1701_01607_gb300 import synth
    m.load(build_if_missing=True)
    out = {"metric": "iterations and seconds to E_inf <= 1e-3; sweep ms per launch",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "64x64x129 two-level box, eps 1e-4, sigma 0.3, seed 1, "
                                  "17 frequencies on [-5, 5]", "nu": NU, "target_e_inf": 1e-3}}
    for gamma in (0.0, 0.5, 1.0):
        atom = synth.TwoLevelAtom(n_freq=17, x_max=5.0, gamma_prd=gamma)
        atm, _ = synth.stratified_two_level(GRID[0], GRID[1], GRID[2], eps=1e-4, sigma=0.3,
                                            seed=1, atom=atom)
        ref = m.mg3d_create(atm, atom, n_grids=3, **NU)
        m.mg3d_fas_solve(ref, 1e-9, 400, n_grids=3)
        n_ref = m.mg3d_get_populations(ref, 3)
        m.mg3d_destroy(ref)
        row = {"fas": _to_target(m, lambda: m.mg3d_create(atm, atom, n_grids=3, **NU), 3, n_ref,
                                 lambda h, it: m.mg3d_fas_vcycle(h, it == 0), 60),
               "mali": _to_target(m, lambda: m.mg3d_create(atm, atom, n_grids=1, **NU), 1, n_ref,
                                  lambda h, it: m.mg3d_mali_sweep(h, 1, 1), 3000)}
        for prec, pname in ((m.MG3D_PREC_F64, "f64"), (m.MG3D_PREC_F32, "f32")):
            h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=prec, **NU)
            try:
                m.mg3d_autotune(h)
                m.mg3d_set_timing(h, True)
                m.mg3d_reset_counters(h)
                for _ in range(5):
                    m.mg3d_formal_solve(h, 1, want=False)
                c = m.mg3d_get_counters(h)
                row[f"sweep_{pname}"] = {
                    "ms": round(c["fs_kernel_ms"] / c["fs_timed_launches"], 3),
                    "shape": list(m.mg3d_get_fs_config(h, 1))}
            finally:
                m.mg3d_destroy(h)
        out[f"gamma_{gamma:g}"] = row
    return out


def run_interpolation(args):
    """The Hermite options of Sec. 3 and Sec. 4.5 on the 64x64x129 two-level
    box (eps = 1e-4; rough sigma = 0.3 and smooth sigma = 0), FP64:
    iterations and seconds to E_inf <= 1e-3 for MALI and 3-grid FAS with
    trilinear or Hermite prolongation, each upwind scheme against its own
    FAS reference converged to C < 1e-9; then the autotuned sweep time of
    each upwind scheme (two-level box, FP64 and FP32; 6-level atom with 120
    frequencies on a 64x64x129 chromosphere).  Opt-in, --interp-experiment;
    prints one JSON line."""
    from paper_1701_01607_gb300 import mg3d as m
    from paper_1701_01607_gb300 import synth
    m.load(build_if_missing=True)
    out = {"metric": "iterations and seconds to E_inf <= 1e-3; sweep ms per launch",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
           "data": "synthetic", "config": {"nu": NU, "target_e_inf": 1e-3}}

    for name, sigma in (("rough", 0.3), ("smooth", 0.0)):
        atm, atom = synth.stratified_two_level(GRID[0], GRID[1], GRID[2], eps=1e-4,
                                               sigma=sigma, seed=1)
        for sc in (0, 1):
            ref = m.mg3d_create(atm, atom, n_grids=3, sc_interp=sc, **NU)
            m.mg3d_fas_solve(ref, 1e-9, 400, n_grids=3)
            n_ref = m.mg3d_get_populations(ref, 3)
            m.mg3d_destroy(ref)
            row = {}
            for interp in (0, 1):
                row[f"fas_{'hermite' if interp else 'trilinear'}"] = _to_target(
                    m, lambda: m.mg3d_create(atm, atom, n_grids=3, sc_interp=sc,
                                             interpolation=interp, **NU),
                    3, n_ref, lambda h, it: m.mg3d_fas_vcycle(h, it == 0), 60)
            row["mali"] = _to_target(
                m, lambda: m.mg3d_create(atm, atom, n_grids=1, sc_interp=sc, **NU),
                1, n_ref, lambda h, it: m.mg3d_mali_sweep(h, 1, 1), 2000)
            out[f"{name}_upwind_{'hermite' if sc else 'linear'}"] = row

    sweeps = {}
    atm, atom = synth.stratified_two_level(GRID[0], GRID[1], GRID[2], eps=1e-4, sigma=0.3,
                                           seed=1)
    for prec, pname in ((m.MG3D_PREC_F64, "f64"), (m.MG3D_PREC_F32, "f32")):
        for sc in (0, 1):
            h = m.mg3d_create(atm, atom, n_grids=1, fs_prec=prec, sc_interp=sc, **NU)
            try:
                m.mg3d_autotune(h)
                m.mg3d_set_timing(h, True)
                m.mg3d_reset_counters(h)
                for _ in range(5):
                    m.mg3d_formal_solve(h, 1, want=False)
                c = m.mg3d_get_counters(h)
                sweeps[f"two_level_{pname}_{'hermite' if sc else 'linear'}"] = {
                    "ms": round(c["fs_kernel_ms"] / c["fs_timed_launches"], 3),
                    "shape": list(m.mg3d_get_fs_config(h, 1))}
            finally:
                m.mg3d_destroy(h)
    ml_atom = synth.hydrogen_like_atom(line_freq=20, cont_freq=4, seed=2)
    ml_atm = synth.chromosphere(64, 64, 129, ml_atom, seed=2)
    for prec, pname in ((m.MG3D_PREC_F32, "f32"), (m.MG3D_PREC_F64, "f64")):
        for sc in (0, 1):
            h = m.mg3d_create_ml(ml_atm, ml_atom, n_grids=1, fs_prec=prec, sc_interp=sc)
            try:
                m.mg3d_autotune(h)
                m.mg3d_set_timing(h, True)
                m.mg3d_reset_counters(h)
                for _ in range(3):
                    m.mg3d_formal_solve_ml(h, 1)
                c = m.mg3d_get_counters(h)
                sweeps[f"six_level_{pname}_{'hermite' if sc else 'linear'}"] = {
                    "ms": round(c["fs_kernel_ms"] / c["fs_timed_launches"], 3),
                    "gunits_s": round(c["fs_units"] / (c["fs_kernel_ms"] * 1e-3) / 1e9, 2),
                    "shape": list(m.mg3d_get_ml_shape(h, 1))}
            finally:
                m.mg3d_destroy(h)
    out["sweeps"] = sweeps
    return out


def run_experiments(args):
    """Synthetic analogues of the paper's restriction and grid-count tests
    (Sec. 4.3, Sec. 4.4): FAS from the zero-radiation start until the true
    error E_inf against a converged reference is <= 1e-3 (cap 60 cycles), for
    full weighting, half weighting and injection on 2, 3 and 4 grids, on the
    rough 64x64x129 box (log-normal sigma = 0.3) and on a smooth one
    (sigma = 0, horizontally homogeneous); FP64.  Opt-in, --experiments."""
    import torch

    from paper_1701_01607_gb300 import mg3d as m
    from paper_1701_01607_gb300 import synth
    m.load(build_if_missing=True)
    stream = torch.cuda.Stream()
    restrictions = (("full", m.MG3D_RESTRICT_FULL), ("half", m.MG3D_RESTRICT_HALF),
                    ("injection", m.MG3D_RESTRICT_INJECT))
    out = {"metric": "V-cycles and seconds to E_inf <= 1e-3 (FAS, two-level atom, 64x64x129)",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
           "data": "synthetic", "config": {"nu": NU, "target_e_inf": 1e-3, "cap_cycles": 60}}
    for name, sigma in (("rough", 0.3), ("smooth", 0.0)):
        atm, atom = synth.stratified_two_level(GRID[0], GRID[1], GRID[2], eps=1e-4,
                                               sigma=sigma, seed=1)
        ref = m.mg3d_create(atm, atom, n_grids=3, fs_prec=m.MG3D_PREC_F64, **NU)
        m.mg3d_set_stream(ref, stream.cuda_stream)
        m.mg3d_fas_solve(ref, 1e-9, 400, n_grids=3)
        n_ref = m.mg3d_get_populations(ref, 3)
        m.mg3d_destroy(ref)
        rows = {}
        for rname, rmode in restrictions:
            for grids in (2, 3, 4):
                h = m.mg3d_create(atm, atom, n_grids=grids, fs_prec=m.MG3D_PREC_F64,
                                  restriction=rmode, **NU)
                m.mg3d_set_stream(h, stream.cuda_stream)
                secs, errs = 0.0, []
                try:
                    for cyc in range(60):
                        t0 = time.perf_counter()
                        m.mg3d_fas_vcycle(h, cyc == 0)
                        secs += time.perf_counter() - t0
                        n = m.mg3d_get_populations(h, grids)
                        errs.append(float(np.max(np.abs(n - n_ref) / np.abs(n_ref))))
                        if errs[-1] <= 1e-3:
                            break
                    status = "ok" if errs[-1] <= 1e-3 else "no"
                except m.MG3DError as e:
                    status = f"error: {e}"
                finally:
                    m.mg3d_destroy(h)
                rows[f"{rname}_{grids}grids"] = {
                    "reached": status, "cycles": len(errs), "seconds": round(secs, 3),
                    "e_inf": [float(f"{x:.3g}") for x in errs[:8]] + (
                        [float(f"{errs[-1]:.3g}")] if len(errs) > 8 else [])}
        out[name] = rows
    return out


def run_chromosphere(args):
    """MALI, FAS and FMG from the zero-radiation start to C < 1e-3 on the
    128x128x257 chromosphere (``--chromo-size``) with the 6-level atom at 600
    frequencies (FP32 formal solution, FP64 rates, 3 grids,
    (nu_0, nu_1, nu_2, nu_3) = (20, 4, 8, 32), sweep shapes autotuned first;
    opt-in, --chromosphere).  ``--scattering`` sets the grey background
    scattering opacity in units of the thermal continuum opacity (Sec. 4.8),
    ``--ground-collisions`` scales the collisions out of the ground level
    (default 1e-3: scattering-dominated resonance lines, so that MALI's
    spectral radius is close to one as in the paper's chromospheres; 1 gives
    collision-dominated lines that MALI solves in a few sweeps).
    Prints one JSON line."""
    from paper_1701_01607_gb300 import mg3d as m
    from paper_1701_01607_gb300 import synth
    m.load(build_if_missing=True)
    nx, ny, nz = (int(v) for v in args.chromo_size.split(","))
    atom = synth.hydrogen_like_atom(line_freq=100, cont_freq=20, seed=2)
    atm = synth.chromosphere(nx, ny, nz, atom, seed=2, ground_collisions=args.ground_collisions,
                             scattering=args.scattering)
    params = dict(fs_prec=m.MG3D_PREC_F32, nu_fmg=16, nu0=20, nu1=4, nu2=8, nu3=32)
    units_fine = nx * ny * nz * 24 * 600
    size = f"{nx}x{ny}x{nz}"
    out = {"metric": f"time to C < 1e-3, 6-level atom (600 frequencies), {size}",
           "unit": "s", "higher_is_better": False, "n_gpus": 1,
           "dtype": "f32 formal solution, f64 rates", "data": "synthetic",
           "config": {"workload": f"chromosphere {size}, 6-level atom, seed 2",
                      "scattering": args.scattering,
                      "ground_collisions": args.ground_collisions, **params}}
    for method, grids, fn, cap in (("fas", 3, m.mg3d_fas_solve, 40),
                                   ("fmg", 3, m.mg3d_fmg_solve, 40),
                                   ("mali", 1, m.mg3d_mali_solve, 400)):
        h = m.mg3d_create_ml(atm, atom, n_grids=grids, **params)
        try:
            m.mg3d_autotune(h)
            m.mg3d_set_timing(h, True)
            m.mg3d_reset_counters(h)
            try:
                st = fn(h, 1e-3, cap, n_grids=grids)
            except m.MG3DError as e:
                out[method] = {"reached": False, "error": str(e)}
                continue
            c = m.mg3d_get_counters(h)
            n = m.mg3d_get_populations(h, grids)
        finally:
            m.mg3d_destroy(h)
        out[method] = {"seconds": round(st["seconds"], 2), "iterations": st["iterations"],
                       "fine_fs_equivalents": round(st["fine_fs_equivalents"], 1),
                       "fs_gunits_s": round(c["fs_units"] / (c["fs_kernel_ms"] * 1e-3) / 1e9, 2),
                       "negatives": st["negatives"],
                       "conservation": float(np.max(np.abs(n.sum(axis=0) / atm.n_tot - 1)))}
    out["value"] = out["fas"].get("seconds")
    out["fine_fs_units"] = units_fine
    return out


CONFIG4_PARAMS = dict(nu_fmg=16, nu0=20, nu1=4, nu2=8, nu3=32)


def config4_atmosphere(size, freqs, ground_collisions=1e-3):
    """The 6-level chromosphere of config 4: 256x256x385 nodes (``size``),
    horizontal spacing 24 km taken as the length unit, heights stretched from
    13 km in the middle to 60 km at the ends (the paper's Model 2 pattern),
    seed 3; ``freqs`` (line, continuum) frequencies per transition; the
    collisions out of the ground level scaled by ``ground_collisions`` (the
    resonance lines scattering-dominated, as in the other chromosphere runs)."""
    from paper_1701_01607_gb300 import synth
    nx, ny, nz = size
    atom = synth.hydrogen_like_atom(line_freq=freqs[0], cont_freq=freqs[1], seed=2)
    z = synth.stretched_heights(nz, 13.0 / 24.0, 60.0 / 24.0)
    return synth.chromosphere(nx, ny, nz, atom, seed=3, z=z, dx=1.0,
                              ground_collisions=ground_collisions), atom


def run_config4(args):
    """Full multigrid on the config-4 chromosphere with 4 grids and
    (nu_FMG, nu_0, nu_1, nu_2, nu_3) = (16, 20, 4, 8, 32) (Table 1, Model 2
    row), the FP32 formal solution (FP64 rates) against FP64 throughout: the
    error of FP32 against FP64 on each grid after each FMG stage (Sec. 2.3:
    stage 1 solves grid 1, stage k interpolates to grid k and, below the
    finest grid, runs a V-cycle there) and after the same number of finest-grid
    V-cycles (--c4-f64-cycles, FP64 being the costlier run); FP32 then goes on
    to C < 1e-3 (time to solution).  Optionally (--c4-mali) FP32 MALI to the
    same rule.  Opt-in (--config4); --c4-size and --c4-freqs shrink it.
    Prints one JSON line."""
    from paper_1701_01607_gb300 import mg3d as m
    m.load(build_if_missing=True)
    size = tuple(int(v) for v in args.c4_size.split(","))
    freqs = tuple(int(v) for v in args.c4_freqs.split(","))
    t0 = time.perf_counter()
    atm, atom = config4_atmosphere(size, freqs, args.ground_collisions)
    build_s = time.perf_counter() - t0
    L = 4
    ncmp = args.c4_f64_cycles
    runs = {}
    for prec, key in ((m.MG3D_PREC_F64, "f64"), (m.MG3D_PREC_F32, "f32")):
        if key == "f64" and args.c4_no_f64:
            continue
        max_cycles = ncmp if key == "f64" else args.c4_max_cycles
        h = m.mg3d_create_ml(atm, atom, n_grids=L, fs_prec=prec, **CONFIG4_PARAMS)
        try:
            t0 = time.perf_counter()
            m.mg3d_autotune(h)
            tune_s = time.perf_counter() - t0
            stages, pops = [], []
            m.mg3d_reset_counters(h)
            t_all = time.perf_counter()
            for k in range(1, L + 1):
                t0 = time.perf_counter()
                m.mg3d_fmg_stage(h, k)
                stages.append(round(time.perf_counter() - t0, 3))
                pops.append(m.mg3d_get_populations(h, k))
            cs, cyc, at_cmp, cycle_s = [], 0, None, []
            while cyc < max_cycles:
                t0 = time.perf_counter()
                cs.append(m.mg3d_fas_vcycle(h, cyc == 0))
                cycle_s.append(round(time.perf_counter() - t0, 2))
                cyc += 1
                if cyc == ncmp:
                    at_cmp = m.mg3d_get_populations(h, L)
                if cs[-1] < 1e-3:
                    break
            secs = time.perf_counter() - t_all
            units = m.mg3d_get_counters(h)["fs_units"]
            final = m.mg3d_get_populations(h, L)
        finally:
            m.mg3d_destroy(h)
        r = {"autotune_s": round(tune_s, 1), "stage_seconds": stages, "cycle_seconds": cycle_s,
             "cycles": cyc, "C": [float(c) for c in cs], "seconds": round(secs, 2),
             "reached_tol": bool(cs and cs[-1] < 1e-3),
             "fine_fs_equivalents": round(units / (np.prod(size) * 24 * n_freq_of(atom)), 1),
             "conservation": float(np.max(np.abs(final.sum(axis=0) / atm.n_tot - 1)))}
        print(json.dumps({"config4_partial": key, **r}), file=sys.stderr, flush=True)
        runs[key] = dict(r, pops=pops, at_cmp=at_cmp)
    out = {"metric": "config 4: FMG, FP32 formal solution against FP64, error per grid",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "chromosphere %dx%dx%d, 6-level atom, %d frequencies, stretched z "
                                  "(13-60 km, dx = 24 km), seed 3, ground collisions x %g"
                                  % (size + (n_freq_of(atom), args.ground_collisions)),
                      "n_grids": L, **CONFIG4_PARAMS},
           "atmosphere_build_s": round(build_s, 1)}
    for key, r in runs.items():
        out[key] = {k: v for k, v in r.items() if k not in ("pops", "at_cmp")}
    if "f64" in runs:
        a, b = runs["f32"], runs["f64"]
        out["f32_vs_f64_e_inf_by_stage"] = {
            f"stage {k + 1} (grid {k + 1})": float(np.max(np.abs(a["pops"][k] - b["pops"][k])
                                                       / np.abs(b["pops"][k])))
            for k in range(L)}
        if a["at_cmp"] is not None and b["at_cmp"] is not None:
            out[f"f32_vs_f64_e_inf_after_{ncmp}_cycles"] = float(
                np.max(np.abs(a["at_cmp"] - b["at_cmp"]) / np.abs(b["at_cmp"])))
    if args.c4_mali:
        h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=m.MG3D_PREC_F32, **CONFIG4_PARAMS)
        try:
            m.mg3d_autotune(h)
            try:
                st = m.mg3d_mali_solve(h, 1e-3, args.c4_mali_max)
                out["mali_f32"] = {"seconds": round(st["seconds"], 2),
                                   "iterations": st["iterations"],
                                   "fine_fs_equivalents": round(st["fine_fs_equivalents"], 1)}
            except m.MG3DError as e:
                out["mali_f32"] = {"reached": False, "error": str(e)}
        finally:
            m.mg3d_destroy(h)
    out["value"] = out["f32"]["seconds"]
    return out


def n_freq_of(atom):
    """Frequencies of a multi-level atom: every line's and continuum's."""
    return sum(t.n_freq for t in atom.lines) + sum(t.n_freq for t in atom.continua)


def run_profile_ml(prec_name, launches, shape=""):
    """A few multi-level formal solutions for ncu: the 6-level atom with 120
    frequencies (lines 5 x 20, continua 5 x 4) on a 64x64x129 chromosphere,
    about 2 GB on the device in FP32.  ``shape`` "bands,rays_per_block,threads"
    fixes the multi-level sweep's shape (e.g. an autotuned one), and
    "bands,rays_per_block,threads,kind,freq_per_block" its kind as well (1:
    the shifted-plane form); no tuning runs here, so every sweep launch is a
    profiled one."""
    from paper_1701_01607_gb300 import mg3d as m
    from paper_1701_01607_gb300 import synth
    m.load(build_if_missing=True)
    atom = synth.hydrogen_like_atom(line_freq=20, cont_freq=4, seed=2)
    atm = synth.chromosphere(64, 64, 129, atom, seed=2)
    prec = m.MG3D_PREC_F64 if prec_name == "f64" else m.MG3D_PREC_F32
    h = m.mg3d_create_ml(atm, atom, n_grids=1, fs_prec=prec)
    try:
        if shape:
            v = [int(x) for x in shape.split(",")]
            if len(v) == 5:
                m.mg3d_set_ml_shape_ex(h, 1, *v)
            else:
                m.mg3d_set_ml_shape(h, 1, *v)
        for _ in range(launches):
            m.mg3d_mali_sweep(h, 1, 1)
        print("profile case: multi-level", prec_name, m.mg3d_get_ml_shape_ex(h, 1),
              "chunk", m.mg3d_get_ml_chunk(h), flush=True)
    finally:
        m.mg3d_destroy(h)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--no-tts", action="store_true", help="skip time-to-solution runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the FP32 sweep on 128x128 planes")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default sweep shapes")
    ap.add_argument("--shapes", default="",
                    help='sweep shapes instead of autotuning, as a bench line reports them: '
                         '{"f64": {"1": [ng, bands, threads, lean, stage], ...}, "f32": {...}}')
    ap.add_argument("--profile-sweep", choices=["f64", "f32"],
                    help="only run a few finest-grid formal solutions (for ncu)")
    ap.add_argument("--experiments", action="store_true",
                    help="run the restriction / grid-count experiments instead")
    ap.add_argument("--chromosphere", action="store_true",
                    help="time MALI, FAS and FMG on the 128x128x257 6-level chromosphere instead")
    ap.add_argument("--prd-experiment", action="store_true",
                    help="partial redistribution against complete redistribution")
    ap.add_argument("--velocity-experiment", action="store_true",
                    help="a moving atmosphere against a static one")
    ap.add_argument("--interp-experiment", action="store_true",
                    help="the Hermite interpolation options against the linear ones")
    ap.add_argument("--scattering-experiment", action="store_true",
                    help="MALI and FAS to E_inf <= 1e-3 against background scattering strength")
    ap.add_argument("--chromo-size", default="128,128,257", help="nx,ny,nz of --chromosphere")
    ap.add_argument("--config4", action="store_true",
                    help="FMG on the 256x256x385 chromosphere, FP32 against FP64 per grid")
    ap.add_argument("--c4-size", default="256,256,385", help="nx,ny,nz of --config4")
    ap.add_argument("--c4-freqs", default="100,20",
                    help="frequencies per line and per continuum of --config4")
    ap.add_argument("--c4-max-cycles", type=int, default=20)
    ap.add_argument("--c4-no-f64", action="store_true", help="--config4 without the FP64 run")
    ap.add_argument("--c4-f64-cycles", type=int, default=2,
                    help="finest-grid V-cycles of the FP64 run of --config4 (FP32 compared there)")
    ap.add_argument("--c4-mali", action="store_true", help="--config4 with an FP32 MALI run")
    ap.add_argument("--c4-mali-max", type=int, default=300)
    ap.add_argument("--scattering", type=float, default=0.0,
                    help="--chromosphere: background scattering opacity / thermal continuum opacity")
    ap.add_argument("--ground-collisions", type=float, default=1e-3,
                    help="--chromosphere: factor on the collisions out of the ground level")
    ap.add_argument("--batch", action="store_true",
                    help="time batched V-cycles of the 32-atmosphere batch instead")
    ap.add_argument("--profile-ml", choices=["f64", "f32"],
                    help="only run a few multi-level MALI sweeps (for ncu)")
    ap.add_argument("--profile-launches", type=int, default=3)
    ap.add_argument("--peaks", action="store_true",
                    help="only measure the FP32/MUFU/FP64 peak rates (mg3d_probe_alu_peaks)")
    ap.add_argument("--profile-shape", default="",
                    help="ng,bands,threads[,lean[,stage]] of the profiled sweep, or "
                         "bands,rays_per_block,threads with --profile-ml")
    args = ap.parse_args()
    if args.peaks:
        from paper_1701_01607_gb300 import mg3d as m
        m.load(build_if_missing=True)
        print(json.dumps({k: v / 1e12 for k, v in m.mg3d_probe_alu_peaks(5).items()}), flush=True)
        return
    if args.profile_sweep:
        run_profile_case(args.profile_sweep, args.profile_launches, args.profile_shape)
        return
    if args.profile_ml:
        run_profile_ml(args.profile_ml, args.profile_launches, args.profile_shape)
        return
    if args.batch:
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.config4:
        print(json.dumps(run_config4(args)), flush=True)
        return
    if args.prd_experiment:
        print(json.dumps(run_prd(args)), flush=True)
        return
    if args.velocity_experiment:
        print(json.dumps(run_velocity(args)), flush=True)
        return
    if args.interp_experiment:
        print(json.dumps(run_interpolation(args)), flush=True)
        return
    if args.scattering_experiment:
        print(json.dumps(run_scattering(args)), flush=True)
        return
    if args.chromosphere:
        print(json.dumps(run_chromosphere(args)), flush=True)
        return
    if args.experiments:
        print(json.dumps(run_experiments(args)), flush=True)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
