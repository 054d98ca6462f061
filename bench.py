"""Benchmark of libsfchem: chem+thermal cell-updates/s of the per-cell
thermochemical update (SFUMATO#, arXiv 2604.21438, Sec. 2.2.8), mixed
precision batched against plain FP64 on the same GPU, at the error stated
against the FP64 CPU oracle.

A step is one call that advances every cell of the workload by its hydro
time step (all substeps of all cells).  Default workload: the GMC-like
256^3 grid (16.8M cells, dt = 1e3 yr, C_d = 1e6 erg/g/K) in 16^3 blocks,
solved by the persistent batched kernel in mixed precision; the plain FP64
path runs the same workload.  Inputs (2.4 GB of state) are larger than L2
and are reset from a pristine device copy before every step (outside the
timed events; the copy also evicts L2).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import inputs  # noqa: E402

METRIC = "chem+thermal cell-updates/s: mixed/batched vs plain FP64 at stated error"
YR = inputs.YR

# Executed FP work per cell-substep of the solver kernels: the FP
# instructions that ncu counts per launch (FMA = 2 flops, add/mul = 1),
# divided by the substeps of that launch, on the first 512 blocks of the
# GMC-like 256^3 workload (2,097,152 cells, dt = 1e3 yr, C_d = 1e6);
# profiles/sfchem_li_mixed_gmc256.md, profiles/sfchem_li_fp64_gmc256.md.
PROFILE_SOURCE = "ncu capture of the GMC-like 256^3 workload, first 512 blocks (profiles/)"
WORK_PER_SUBSTEP = {
    "mixed": {"fp32_flops": 1285.2, "fp64_flops": 30.2},
    "fp64": {"fp32_flops": 1.6, "fp64_flops": 1964.4},
}
# DRAM bytes per cell of one solver launch (same captures, 2,097,152 cells:
# 282.0 MB mixed, 263.7 MB FP64).
DRAM_BYTES_PER_CELL = {"mixed": 282.03e6 / 2097152, "fp64": 263.72e6 / 2097152}
# DRAM bytes per cell of the photon kernel (ncu, one launch on the full
# GMC-like grid: 48.0 B read, 14.7 B written; profiles/sfchem_photon_kernel_gmc256.md)
PHOTON_DRAM_BYTES_PER_CELL = (805.33e6 + 246.62e6) / 16777216
# GB300 ALU peaks from unit counts and the SM clock: 152 SMs; FP32 128
# lanes/SM (256 flops/clk); FP64 2 DFMA/clk/SM (4 flops/clk) -- the
# "peak_sustained" of the FP64 pipe that ncu reports, 1.26 TFLOP/s at 2.07 GHz.
N_SM = 152
FP32_FLOP_PER_SM_CLK = 256.0
FP64_FLOP_PER_SM_CLK = 4.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--workload", default="gmc256", choices=("gmc256", "grf128", "amr3000", "uniform4096", "be"))
    p.add_argument("--Z", type=float, default=1.0, choices=(1.0, 1e-2, 1e-4),
                   help="metallicity of the Bonnor-Ebert sphere workload (Z / Z_sun)")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison leg")
    p.add_argument("--no-ff", action="store_true", help="skip the mixed leg with the FP32 error-free refinement")
    p.add_argument("--no-nr", action="store_true", help="skip the Newton-Raphson reference leg")
    p.add_argument("--sweep", action="store_true", help="run the dt x C_d sweep on the GRF 128^3 grid instead")
    p.add_argument("--sweep-precision", default="fp64", choices=("fp64", "mixed"))
    p.add_argument("--sweep-z", action="store_true",
                   help="run the metallicity / C_d sweep on the Bonnor-Ebert sphere instead")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle legs (error check, cpu_baseline)")
    p.add_argument("--sample", type=int, default=4096, help="cells checked against the oracle")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target wall time of the cpu_baseline")
    p.add_argument("--slice-blocks", type=int, default=0,
                   help="use only the first N blocks of the workload (small cases for profiling)")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg through host buffers")
    return p.parse_args()


# ------------------------------------------------------------------ workloads
def make_workload(name: str, rank: int = 0, Z: float = 1.0):
    """(cells, block_offset, block_dt, cd_factor, description)"""
    if name == "be":
        cells, off, lvl = inputs.cells_be(Z)
        bdt = np.full(len(off) - 1, inputs.be_dt())
        return cells, off, bdt, 1e3, dict(
            workload="initial Bonnor-Ebert sphere, nested grids l_max = 2 (1408 blocks of 8^3)",
            cells=len(cells["n_H"]), Z=Z, dt_yr=inputs.be_dt() / YR, cd_factor=1e3, C_d=1e7,
            blocks=len(bdt), block_cells=512)
    if name == "gmc256":
        cells = inputs.cells_gmc(256, seed=1005 + rank)
        cells, off = inputs.block_major(cells, 256, 16)
        bdt = np.full(len(off) - 1, 1e3 * YR)
        return cells, off, bdt, 100.0, dict(
            workload="GMC-like 256^3 grid in 16^3 blocks", cells=len(cells["n_H"]), dt_yr=1e3,
            cd_factor=100.0, blocks=len(bdt), block_cells=4096)
    if name == "grf128":
        cells = inputs.cells_grf(128, seed=1002 + rank)
        cells, off = inputs.block_major(cells, 128, 16)
        bdt = np.full(len(off) - 1, 1e3 * YR)
        return cells, off, bdt, 1.0, dict(workload="GRF 128^3 grid in 16^3 blocks", cells=len(cells["n_H"]),
                                          dt_yr=1e3, cd_factor=1.0, blocks=len(bdt), block_cells=4096)
    if name == "amr3000":
        cells, off, bdt, lvl = inputs.cells_amr(seed=1004 + rank)
        return cells, off, bdt, 100.0, dict(workload="AMR 3000 blocks of 8^3, levels 0-6, dt_l = 1e3 yr / 2^l",
                                            cells=len(cells["n_H"]), cd_factor=100.0, blocks=len(bdt),
                                            block_cells=512)
    cells = inputs.cells_uniform(4096, seed=1001 + rank)
    off = np.array([0, 4096], np.int64)
    return cells, off, np.array([1e3 * YR]), 1.0, dict(workload="4096 independent cells (one 16^3 block)",
                                                       cells=4096, dt_yr=1e3, cd_factor=1.0, blocks=1,
                                                       block_cells=4096)


# -------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def microbench_fma():
    """Measured FP64 / FP32 FMA throughput (FLOP/s) of this GPU."""
    import ctypes
    from paper_2604_21438_gb300 import _build
    _build.build()
    L = ctypes.CDLL(_build.BENCH_LIB)
    out = {}
    for name in ("fp64", "fp32"):
        f = getattr(L, f"sfbench_fma_{name}")
        fl, ms = ctypes.c_double(), ctypes.c_float()
        iters = 2000 if name == "fp64" else 20000
        if f(iters, ctypes.byref(fl), ctypes.byref(ms)) == 0:
            out[name] = fl.value
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2604_21438_gb300 as sf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1 and args.workload == "gmc256":
        cells, off, bdt, cd, desc = sharded_gmc(args, rank, world, dev)
    else:
        cells, off, bdt, cd, desc = make_workload(args.workload, rank, args.Z)
    if args.slice_blocks:
        nb = min(args.slice_blocks, len(bdt))
        cells = inputs.subset(cells, np.arange(int(off[nb])))
        off, bdt = off[:nb + 1], bdt[:nb]
        desc = dict(desc, cells=int(off[-1]), blocks=nb, slice=f"first {nb} blocks")
    Z = desc.get("Z", 1.0)
    n = len(cells["n_H"])
    stream = torch.cuda.current_stream()

    d = sf.to_device(cells, dev)
    pristine = {k: d[k].clone() for k in sf.STATE_FIELDS}

    def reset():
        for k in sf.STATE_FIELDS:
            d[k].copy_(pristine[k], non_blocking=True)

    def timed_leg(solver, steps, warmup, reset_each=True):
        for _ in range(warmup):
            reset()
            solver.step_batched(d, off, bdt, cd)
        torch.cuda.synchronize()
        solver.stats_reset()
        times = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            if reset_each:
                reset()
            ev[i][0].record(stream)
            solver.step_batched(d, off, bdt, cd)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - t0
        times = [a.elapsed_time(b) for a, b in ev]
        st = solver.stats()
        return float(np.mean(times)), wall, st

    res = {}
    # ---- mixed precision, batched (the headline)
    sm = sf.Solver("mixed", Z=Z)
    if not args.no_autotune:
        reset()
        sm.autotune(d, off, bdt, cd)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms_m, wall_m, st_m = timed_leg(sm, args.steps, args.warmup)
    clk = clocks.stop()
    out_m = sf.to_host({k: d[k] for k in sf.STATE_FIELDS + ("status", "n_sub")})
    res["mixed"] = dict(ms=ms_m, wall=wall_m, stats=st_m, launch=sm.get_launch())
    # ---- photon consumption after the update (sfchem_photon_update), on the
    # updated state; HBM-bound: 6 FP64 reads and 2 FP64 writes per cell
    g_out, e_out = torch.empty_like(d["G0"]), torch.empty_like(d["n_EUV"])
    for _ in range(3):
        sf.photon_update(d, float(bdt[0]), G0_out=g_out, n_euv_out=e_out)
    torch.cuda.synchronize()
    pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a0, b0 in pe:
        a0.record(stream)
        sf.photon_update(d, float(bdt[0]), G0_out=g_out, n_euv_out=e_out)
        b0.record(stream)
    torch.cuda.synchronize()
    res["photon"] = dict(ms=float(np.mean([a0.elapsed_time(b0) for a0, b0 in pe])))
    del g_out, e_out
    # ---- mixed precision with the error-free FP32 refinement residual
    out_ff = None
    if not args.no_ff:
        sff = sf.Solver("mixed", flags=sf.F_REFINE_FF, Z=Z)
        sff.set_launch(**sm.get_launch())
        ms_ff, wall_ff, st_ff = timed_leg(sff, args.steps, args.warmup)
        out_ff = sf.to_host({k: d[k] for k in sf.STATE_FIELDS + ("status", "n_sub")})
        res["mixed_ff"] = dict(ms=ms_ff, wall=wall_ff, stats=st_ff)
        sff.close()
    # ---- plain FP64, batched, same workload
    out_d = None
    if not args.no_fp64:
        sd = sf.Solver("fp64", Z=Z)
        sd.set_launch(64, 0, 32)           # the fastest of the shapes timed on the GRF 128^3 workload
        k64 = max(1, min(args.steps, 2))   # the slow leg: 1 warm-up, 2 timed steps
        ms_d, wall_d, st_d = timed_leg(sd, k64, 1)
        out_d = sf.to_host({k: d[k] for k in sf.STATE_FIELDS + ("status", "n_sub")})
        res["fp64"] = dict(ms=ms_d, wall=wall_d, stats=st_d, steps=k64, warmup=1, launch=sd.get_launch())
        sd.close()
    # ---- the Newton-Raphson reference solver (Sec. 2.2.8) on the same workload
    if not args.no_nr and np.all(bdt == bdt[0]):
        snr = sf.Solver("fp64", n_sub_max=2000, Z=Z)
        for _ in range(1):
            reset()
            snr.step_nr(d, float(bdt[0]), cd)
        torch.cuda.synchronize()
        snr.stats_reset()
        times = []
        for _ in range(2):
            reset()
            a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            snr.step_nr(d, float(bdt[0]), cd)
            b0.record(stream)
            torch.cuda.synchronize()
            times.append(a0.elapsed_time(b0))
        stn = snr.stats()
        res["nr"] = dict(ms=float(np.mean(times)), stats=stn)
        snr.close()
    # ---- end to end through the public API with host buffers: sfchem_step_host
    # copies each slice's inputs in and its results out on two streams while
    # the previous slice is solved; the state is reset outside the timed region
    if args.no_e2e:
        e2e_ms = float("nan")
        sm.close()
        return finish_line(args, rank, world, res, clk, n, cells, off, bdt, cd, desc, Z, ms_m, e2e_ms, out_m,
                           out_d, out_ff, 0, 0)
    pristine_h = {k: torch.as_tensor(cells[k]).pin_memory() for k in sf.STATE_FIELDS}
    host = {k: torch.as_tensor(cells[k]).pin_memory() for k in sf.STATE_FIELDS + sf.INPUT_FIELDS}
    host["status"] = torch.empty(n, dtype=torch.uint8).pin_memory()
    h2d = 8 * n * (len(sf.STATE_FIELDS) + len(sf.INPUT_FIELDS))
    d2h = 8 * n * len(sf.STATE_FIELDS) + n
    e2e_times = []
    for i in range(args.warmup + args.steps):
        for k in sf.STATE_FIELDS:
            host[k].copy_(pristine_h[k])
        barrier(world)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sm.step_host(host, off, bdt, cd, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(a.elapsed_time(b))
    e2e_ms = float(np.mean(e2e_times))
    sm.close()
    return finish_line(args, rank, world, res, clk, n, cells, off, bdt, cd, desc, Z, ms_m, e2e_ms, out_m, out_d,
                       out_ff, h2d, d2h)


def finish_line(args, rank, world, res, clk, n, cells, off, bdt, cd, desc, Z, ms_m, e2e_ms, out_m, out_d, out_ff,
                h2d, d2h):
    """The JSON line of our arm from the legs' measurements."""
    # cross-rank aggregation: max time over ranks
    ms_m_max = allreduce_max(ms_m, world)
    e2e_max = allreduce_max(e2e_ms, world)
    total_cells = int(round(allreduce_sum(float(n), world)))
    value = total_cells / (ms_m_max * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_m_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": dict(desc, precision="mixed", path="sfchem_step_batched (persistent kernel, CUDA graph)",
                       l2="inputs (2.4 GB) larger than L2; state reset from a device copy before each step",
                       parallelism=(f"one workload in {world} cost-balanced block ranges (no data-path collective)"
                                    if world > 1 else "one device")),
        "e2e": None if not np.isfinite(e2e_max) else {
            "value": total_cells / (e2e_max * 1e-3), "unit": "cell-updates/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_max,
            "path": "sfchem_step_host: pinned host state, copies overlapped with the solver slice by slice"},
        "gpu_launches": 3 * args.steps,   # per step: schedule kernel, persistent solver kernel, y_H- kernel
        "clocks": clk,
    }
    if "photon" in res:
        peaks, src = measured_peaks()
        ms_p = res["photon"]["ms"]
        gbs = 64.0 * n / (ms_p * 1e-3) / 1e9
        line["photon_update"] = {
            "kernel": "sfchem_photon_kernel", "ms": ms_p, "cells": n,
            "roofline": {"bound": "hbm", "unit": "GB/s", "achieved": gbs, "peak": peaks["hbm_gbs"],
                         "frac": gbs / peaks["hbm_gbs"], "peak_source": src,
                         "bytes_per_cell": 64, "traffic": PHOTON_DRAM_BYTES_PER_CELL * n,
                         "traffic_note": "ncu dram bytes per cell of one full-grid launch x cells"},
            "note": "photon consumption after the update (reading of Sec. 2.2.8), timed alone over 10 launches"}
    if "mixed_ff" in res:
        ms_f_max = allreduce_max(res["mixed_ff"]["ms"], world)
        line["mixed_ff"] = {"value": total_cells / (ms_f_max * 1e-3), "ms_per_step": ms_f_max,
                            "note": "refinement residual by error-free FP32 transformations (SFCHEM_F_REFINE_FF)"}
    if "nr" in res:
        ms_n_max = allreduce_max(res["nr"]["ms"], world)
        stn = res["nr"]["stats"]
        line["nr_fp64"] = {"value": total_cells / (ms_n_max * 1e-3), "ms_per_step": ms_n_max, "steps": 2,
                           "warmup": 1, "substeps_per_cell": stn["substeps"] / max(stn["cells"], 1),
                           "outer_iterations_per_cell": stn["newton_iters"] / max(stn["cells"], 1),
                           "noconv_cells": stn["noconv_cells"],
                           "note": "Newton-Raphson backward-Euler reference (sfchem_step_nr), uniform-dt workloads"}
    if "fp64" in res:
        ms_d_max = allreduce_max(res["fp64"]["ms"], world)
        line["fp64"] = {"value": total_cells / (ms_d_max * 1e-3), "ms_per_step": ms_d_max,
                        "steps": res["fp64"]["steps"], "warmup": 1, "launch": res["fp64"]["launch"],
                        "substeps_per_cell": res["fp64"]["stats"]["substeps"] / max(res["fp64"]["stats"]["cells"], 1)}
        line["speedup_mixed_vs_fp64"] = ms_d_max / ms_m_max
    st = res["mixed"]["stats"]
    line["substeps_per_cell"] = st["substeps"] / max(st["cells"], 1)
    line["step_rejection"] = {"rejected_substeps": st["rejected_substeps"], "step_halvings": st["step_halvings"],
                              "fraction_of_substeps": st["rejected_substeps"] / max(st["substeps"], 1),
                              "note": "substeps redone by the step-rejection reading (mixed leg, all timed steps)"}
    line["tight_fraction"] = st["tight_cells"] / max(st["cells"], 1)
    line["launch"] = res["mixed"]["launch"]
    try:
        line["alu_peaks_microbench_tflops"] = {k: v / 1e12 for k, v in microbench_fma().items()}
    except Exception as exc:  # the measurement is informational
        line["alu_peaks_microbench_tflops"] = {"error": str(exc)}
    # roofline of the dominant kernel (the mixed solver kernel)
    alg = None
    if rank == 0 and not args.no_cpu:
        try:
            alg = algorithmic_work(cells, off, bdt, cd, Z=Z)
        except Exception as exc:  # informational
            alg = None
            line["algorithmic_work_error"] = str(exc)
    line["roofline"] = roofline(res, clk, n, "mixed", alg)
    if "fp64" in res:
        line["roofline_fp64"] = roofline(res, clk, n, "fp64", alg)
    if "nr_fp64" in line and rank == 0 and not args.no_cpu:
        try:
            line["nr_fp64"]["roofline"] = roofline_nr(cells, off, bdt, cd, Z, n, line["nr_fp64"]["ms_per_step"], clk)
        except Exception as exc:  # informational
            line["nr_fp64"]["roofline_error"] = str(exc)
    if alg is not None:
        line["algorithmic_work"] = alg
    if rank == 0 and not args.no_cpu:
        line["error_vs_oracle"] = error_vs_oracle(cells, off, bdt, cd, out_m, out_d, args.sample, out_ff, Z=Z,
                                                   workload=args.workload)
        line["cpu_baseline"] = cpu_baseline(cells, off, bdt, cd, args.cpu_seconds, Z=Z)
    return line


def roofline(res, clk, n_cells, leg="mixed", alg=None):
    """ALU roofline of a solver kernel.

    Primary (achieved / peak / frac): the method's algorithmic work -- the
    oracle's op count W per substep on a sample of this workload
    (algorithmic_work) x the substeps of one launch -- over the launch's
    CUDA-event time, against the peak of the precision the kernel computes
    the method in: FP32 for the mixed kernel, FP64 for the plain one (unit
    counts x max SM clock).  W counts the oracle's dual-number Jacobian and
    its two double-word refinements, about twice what the kernels execute,
    so the plain FP64 kernel can read above 1.0.

    kernel_counted: the FP instructions the kernel executes per substep
    (WORK_PER_SUBSTEP, from the ncu capture of the GMC-like slice) on the
    pipe that binds it (FP64 for both kernels: on GB300 the FP64 rate is
    1/64 of FP32), with the other pipe beside it."""
    st = res[leg]["stats"]
    subs = st["substeps"] / max(st["calls"], 1)
    ms = res[leg]["ms"]
    w = WORK_PER_SUBSTEP[leg]
    f_mhz = clk.get("sm_max_mhz") or 2070.0
    peak64 = N_SM * FP64_FLOP_PER_SM_CLK * f_mhz * 1e6 / 1e12
    peak32 = N_SM * FP32_FLOP_PER_SM_CLK * f_mhz * 1e6 / 1e12
    a64 = w["fp64_flops"] * subs / (ms * 1e-3) / 1e12
    a32 = w["fp32_flops"] * subs / (ms * 1e-3) / 1e12
    kc = {"flops_per_substep": w, "source": PROFILE_SOURCE}
    if a64 / peak64 >= a32 / peak32:
        kc.update(pipe="fp64", achieved=a64, peak=peak64, frac=a64 / peak64,
                  other={"pipe": "fp32", "achieved": a32, "peak": peak32, "frac": a32 / peak32})
    else:
        kc.update(pipe="fp32", achieved=a32, peak=peak32, frac=a32 / peak32,
                  other={"pipe": "fp64", "achieved": a64, "peak": peak64, "frac": a64 / peak64})
    out = {"bound": "alu", "unit": "TFLOP/s", "kernel": f"sfchem_li_{leg}", "substeps_per_launch": subs,
           "kernel_ms": ms, "traffic": DRAM_BYTES_PER_CELL[leg] * n_cells,
           "traffic_note": "dram bytes of one launch: bytes per cell of the ncu capture x cells",
           "algorithmic_bytes": 141 * n_cells}
    peak = peak32 if leg == "mixed" else peak64
    if alg is not None:
        aw = alg["flops_per_substep"] * subs / (ms * 1e-3) / 1e12
        out.update(achieved=aw, peak=peak, frac=aw / peak, pipe="fp32" if leg == "mixed" else "fp64",
                   work="algorithmic: oracle op count W per substep x substeps of the launch",
                   W_flops_per_substep=alg["flops_per_substep"],
                   W_transcendentals_per_substep=alg["transcendentals_per_substep"])
    else:
        # without the oracle (--no-cpu) only the executed-instruction view exists
        out.update(achieved=kc["achieved"], peak=kc["peak"], frac=kc["frac"], pipe=kc["pipe"],
                   work="kernel-counted (no oracle op count in this run)")
    out["kernel_counted"] = kc
    out["peak_source"] = "unit counts x max SM clock (recipe); FMA microbenchmark in alu_peaks_microbench_tflops"
    return out


def oracle_config(Z: float = 1.0):
    import oracle
    c = oracle.default_config()
    c.Z = Z
    return c


# Stated bound on the mixed path's largest relative error per cell (fields
# above 1e-8), per workload; the same bounds as the parity tests.  A cell past
# it is explained when the oracle's own result moves by more than the bound
# for f_chem changed by 1e-3 of itself (a cell at a thermal instability).
STATED_MIXED_MAX = {"gmc256": 2e-5, "amr3000": 2e-4, "be": 2e-4, "uniform4096": 5e-3, "grf128": 5e-3}
FCHEM_PROBE = 1e-3


def fchem_sensitivity(cell, dt, cd, Z=1.0):
    """Largest relative change of the oracle's result (fields above 1e-8)
    for f_chem changed by FCHEM_PROBE of itself, either way."""
    import oracle
    one = {k: np.array([float(v)]) for k, v in cell.items()}
    r0 = oracle.li_step(one, dt, cd, oracle_config(Z))
    out = 0.0
    for sgn in (1.0, -1.0):
        c = oracle_config(Z)
        c.f_chem = c.f_chem * (1.0 + sgn * FCHEM_PROBE)
        r = oracle.li_step(one, dt, cd, c)
        for k in ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H"):
            b = abs(r0[k][0])
            if b > 1e-8:
                out = max(out, abs(r[k][0] - r0[k][0]) / b)
    return out


def error_vs_oracle(cells, off, bdt, cd, out_m, out_d, sample, out_ff=None, Z=1.0, workload=None):
    """Mixed and FP64 results against the oracle on a seeded sample of cells."""
    import oracle
    n = len(cells["n_H"])
    idx = np.sort(np.random.default_rng(123).choice(n, min(sample, n), replace=False))
    blk = np.searchsorted(off, idx, side="right") - 1
    sub = inputs.subset(cells, idx)
    ref = oracle.li_step(sub, bdt[blk], cd, oracle_config(Z))
    out = {"sample_cells": int(idx.size)}
    for name, got in (("mixed", out_m), ("mixed_ff", out_ff), ("fp64", out_d)):
        if got is None:
            continue
        res = {}
        got_yH = 1.0 - 2.0 * got["y_H2"][idx] - got["y_e"][idx]
        for k in ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H"):
            a = got_yH if k == "y_H" else got[k][idx]
            b = ref[k]
            big = np.abs(b) > 1e-8
            d = np.abs(a - b)
            e = d[big] / np.abs(b[big])
            res[k] = {"max": float(e.max()) if e.size else 0.0,
                      "p99": float(np.percentile(e, 99)) if e.size else 0.0,
                      "median": float(np.median(e)) if e.size else 0.0,
                      "abs_max_below_1e-8": float(d[~big].max()) if (~big).any() else 0.0}
        res["n_sub_mismatch"] = int((got["n_sub"][idx] != ref["n_sub"]).sum())
        bound = STATED_MIXED_MAX.get(workload)
        if name == "mixed" and bound is not None:
            worst = np.zeros(idx.size)
            for k in ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H"):
                a = got_yH if k == "y_H" else got[k][idx]
                b = ref[k]
                big = np.abs(b) > 1e-8
                worst = np.maximum(worst, np.where(big, np.abs(a - b) / np.where(big, np.abs(b), 1.0), 0.0))
            over = np.nonzero(worst > bound)[0]
            explained = 0
            for j in over[:32]:
                i = idx[j]
                cell = {k: cells[k][i] for k in inputs.FIELDS}
                if fchem_sensitivity(cell, bdt[blk[j]], cd, Z) > bound:
                    explained += 1
            res["stated_max_bound"] = {"bound": bound, "cells_over": int(over.size),
                                       "checked": int(min(over.size, 32)), "explained_by_fchem_sensitivity": explained}
        out[name] = res
    out["metric"] = "relative error where the oracle's value exceeds 1e-8, absolute error below"
    return out


def cpu_baseline(cells, off, bdt, cd, target_s, Z=1.0):
    """The oracle on the host cores, on a bounded sample of the workload."""
    import oracle
    n = len(cells["n_H"])
    rng = np.random.default_rng(7)
    m = 1024
    while True:
        idx = np.sort(rng.choice(n, min(m, n), replace=False))
        blk = np.searchsorted(off, idx, side="right") - 1
        sub = inputs.subset(cells, idx)
        t0 = time.perf_counter()
        oracle.li_step(sub, bdt[blk], cd, oracle_config(Z))
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or m >= n or m >= (1 << 22):
            break
        m = int(min(n, max(2 * m, m * 0.6 * target_s / max(dt, 1e-3))))
    cores = os.cpu_count()
    out = {"value": idx.size / dt, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
           "sample": f"{idx.size} seeded cells of the workload, one step, {dt:.1f} s wall on {cores} threads"}
    # the same oracle on one host thread, on a quarter of that sample
    q = idx[: max(64, idx.size // max(4, cores // 4))]
    blk = np.searchsorted(off, q, side="right") - 1
    t0 = time.perf_counter()
    oracle.li_step(inputs.subset(cells, q), bdt[blk], cd, oracle_config(Z), n_threads=1)
    d1 = time.perf_counter() - t0
    out["single_thread"] = {"value": q.size / d1, "unit": "cell-updates/s", "cores": 1,
                            "sample": f"{q.size} cells of the same sample, {d1:.1f} s wall on 1 thread"}
    return out


def algorithmic_work(cells, off, bdt, cd, Z=1.0, sample=256):
    """Floating-point work of the method per substep, counted by running the
    oracle's LI step with an op-counting scalar type on a seeded sample of
    the workload (flops: add, mul, div = 1, fma = 2; transcendentals apart)."""
    import oracle
    n = len(cells["n_H"])
    idx = np.sort(np.random.default_rng(31).choice(n, min(sample, n), replace=False))
    blk = np.searchsorted(off, idx, side="right") - 1
    r = oracle.opcount(inputs.subset(cells, idx), bdt[blk], cd, oracle_config(Z))
    per = r["per_substep"]
    sec = {k: sum(v[o] * (2 if o == "fma" else 1) for o in ("add", "mul", "div", "fma")) / max(r["substeps"], 1)
           for k, v in r["counts"].items()}
    return {"flops_per_substep": per["flops"], "transcendentals_per_substep": per["transcendentals"],
            "by_section_flops_per_substep": sec, "sample_cells": int(idx.size), "sample_substeps": r["substeps"],
            "how": "oracle LI step with an op-counting scalar type (oracle/opcount.cpp): forward-mode dual-number "
                   "Jacobian, equilibrated dense 5x5 elimination with two double-word refinements"}


def roofline_nr(cells, off, bdt, cd, Z, n_cells, ms, clk, sample=256):
    """Algorithmic roofline of the Newton-Raphson kernel (FP64): the oracle's
    NR step counted with the op-counting scalar type on a seeded sample of
    the workload (flops per cell), x cells / the kernel's CUDA-event time,
    against the FP64 peak (unit counts x max SM clock)."""
    import oracle
    n = len(cells["n_H"])
    idx = np.sort(np.random.default_rng(37).choice(n, min(sample, n), replace=False))
    blk = np.searchsorted(off, idx, side="right") - 1
    r = oracle.opcount(inputs.subset(cells, idx), bdt[blk], cd, oracle_config(Z), method="nr")
    f_mhz = clk.get("sm_max_mhz") or 2070.0
    peak64 = N_SM * FP64_FLOP_PER_SM_CLK * f_mhz * 1e6 / 1e12
    w = r["per_cell"]["flops"]
    ach = w * n_cells / (ms * 1e-3) / 1e12
    return {"bound": "alu", "unit": "TFLOP/s", "kernel": "sfchem_nr_fp64", "pipe": "fp64", "achieved": ach,
            "peak": peak64, "frac": ach / peak64, "W_flops_per_cell": w,
            "W_transcendentals_per_cell": r["per_cell"]["transcendentals"], "sample_cells": int(idx.size),
            "work": "algorithmic: oracle NR step op count per cell x cells of the launch"}


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle (plain FP64 CPU LI step) timed on the host cores, each step
    one bounded sample of the same workload."""
    import oracle
    cells, off, bdt, cd, desc = make_workload(args.workload, 0, args.Z)
    ocfg = oracle_config(desc.get("Z", 1.0))
    n = len(cells["n_H"])
    rng = np.random.default_rng(99)
    # size the per-step sample so the whole run stays within a few minutes
    probe = np.sort(rng.choice(n, min(2048, n), replace=False))
    t0 = time.perf_counter()
    oracle.li_step(inputs.subset(cells, probe), bdt[np.searchsorted(off, probe, side="right") - 1], cd, ocfg)
    per_cell = (time.perf_counter() - t0) / probe.size
    budget = 120.0 / max(args.steps + args.warmup, 1)
    m = int(min(n, max(1024, budget / max(per_cell, 1e-9))))
    times = []
    for i in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(n, m, replace=False))
        sub = inputs.subset(cells, idx)
        blk = np.searchsorted(off, idx, side="right") - 1
        t0 = time.perf_counter()
        oracle.li_step(sub, bdt[blk], cd, ocfg)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    sec = float(np.mean(times))
    value = m / sec
    cores = os.cpu_count()
    return {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(desc, precision="fp64", path="CPU oracle (OpenMP over cells)",
                           sample_cells_per_step=m),
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{m} seeded cells of the workload per step"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- plumbing
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


_PG = {"on": False}


def init_dist(world, local_rank):
    if world > 1 and not _PG["on"]:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
        _PG["on"] = True


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_sum(x: float, world: int) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def allreduce_max(x: float, world: int) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_slabs(cut, rank: int, slab_blocks: int):
    """The pieces of rank `rank`'s contiguous block range [cut[rank],
    cut[rank + 1]) of a workload made of equal slabs of slab_blocks blocks:
    a list of (slab, first block, end block) with block indices local to the
    slab, in order."""
    lo, hi = int(cut[rank]), int(cut[rank + 1])
    out = []
    b = lo
    while b < hi:
        s = b // slab_blocks
        e = min(hi, (s + 1) * slab_blocks)
        out.append((s, b - s * slab_blocks, e - s * slab_blocks))
        b = e
    return out


def sharded_gmc(args, rank: int, world: int, dev):
    """One workload of `world` GMC-like 256^3 slabs (seeds 1005 + slab), split
    into contiguous block ranges balanced by cost (Sec. 4: the
    thermochemical update runs independently on each device).  Each rank
    first advances its own slab once (untimed) to measure its per-block
    substeps; the costs are gathered, sfchem_partition cuts the block list,
    and each rank assembles its range (whole blocks, from at most a few
    slabs)."""
    import paper_2604_21438_gb300 as sf
    import torch
    slab = {}

    def get(sidx):
        if sidx not in slab:
            c = inputs.cells_gmc(256, seed=1005 + sidx)
            slab[sidx] = inputs.block_major(c, 256, 16)
        return slab[sidx]

    own, off = get(rank)
    nb = len(off) - 1
    bdt = np.full(nb, 1e3 * YR)
    s = sf.Solver("mixed")
    d = sf.to_device(own, dev, outputs=False)
    s.step_batched(d, off, bdt, 100.0)
    torch.cuda.synchronize()
    cost = gather_block_costs(s.block_costs(nb).astype(np.float64), rank * nb, world * nb, world)
    s.close()
    del d
    off_g = np.concatenate([[0], np.cumsum(np.tile(np.diff(off), world))]).astype(np.int64)
    cut = sf.partition(off_g, world, cost)
    parts = []
    offs = [0]
    for sidx, b0, b1 in shard_slabs(cut, rank, nb):
        c, o = get(sidx)
        parts.append(inputs.subset(c, np.arange(int(o[b0]), int(o[b1]))))
        offs.extend((offs[-1] + np.diff(o[b0:b1 + 1])).tolist())
    for k in [k for k in slab if k != rank]:
        del slab[k]
    cells = inputs.concat(*parts)
    loads = [float(cost[cut[r]:cut[r + 1]].sum()) for r in range(world)]
    off_r = np.array(offs, np.int64)
    desc = dict(workload=f"GMC-like 256^3 grid x {world} slabs (one workload) in 16^3 blocks, cost-balanced "
                         f"contiguous block ranges per rank",
                cells=int(off_r[-1]), dt_yr=1e3, cd_factor=100.0, blocks=len(off_r) - 1, block_cells=4096,
                partition={"cut": [int(x) for x in cut], "cost": "substeps per block of a warm-up call",
                           "load_max_over_mean": max(loads) / (sum(loads) / world)})
    return cells, off_r, np.full(len(off_r) - 1, 1e3 * YR), 100.0, desc


def gather_block_costs(mine, lo: int, n_blocks: int, world: int):
    """The per-block costs of one workload, from each rank's costs of its own
    block range [lo, lo + len(mine)): a sum-reduction of zero-padded vectors
    (a host-side exchange between steps, not part of the timed step)."""
    full = np.zeros(n_blocks, np.float64)
    full[lo:lo + len(mine)] = mine
    if world <= 1:
        return full
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.as_tensor(full, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def run_sweep(args):
    """The dt x C_d sweep on the GRF 128^3 grid with the plain FP64 path:
    substep statistics and the deviation of each output from the
    cd_factor = 1 result (one JSON line per sweep)."""
    import torch
    import paper_2604_21438_gb300 as sf
    cells = inputs.cells_grf(128, seed=1002)
    d = sf.to_device(cells)
    pristine = {k: d[k].clone() for k in sf.STATE_FIELDS}
    n = len(cells["n_H"])
    rows = []
    for dt_yr in (1e2, 1e3, 1e4):
        base = None
        for cd in (1.0, 10.0, 100.0, 1000.0):
            for k in sf.STATE_FIELDS:
                d[k].copy_(pristine[k])
            s = sf.Solver(args.sweep_precision)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            s.step(d, dt_yr * YR, cd)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            st = s.stats()
            s.close()
            out = sf.to_host({k: d[k] for k in sf.STATE_FIELDS + ("n_sub", "status")})
            if cd == 1.0:
                base = out
            dev = {}
            for k in ("T_g", "T_d", "y_H2", "y_e"):
                floor = 1e-6 if k.startswith("y_") else 1e-300
                e = np.abs(out[k] - base[k]) / np.maximum(np.abs(base[k]), floor)
                dev[k] = {"max": float(e.max()), "p99": float(np.percentile(e, 99)),
                          "median": float(np.median(e)), "frac_above_1e-3": float((e > 1e-3).mean())}
            ns = out["n_sub"]
            edges = np.array([0, 1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 1 << 30])
            rows.append({"dt_yr": dt_yr, "cd_factor": cd, "C_d": cd * 1e4, "ms": ms,
                         "cell_updates_per_s": n / (ms * 1e-3),
                         "n_sub": {"mean": float(ns.mean()), "p50": float(np.median(ns)),
                                   "p99": float(np.percentile(ns, 99)), "max": int(ns.max()),
                                   "hist_edges": edges.tolist(),
                                   "hist": np.histogram(ns, bins=edges)[0].tolist()},
                         "tight_fraction": st["tight_cells"] / max(st["cells"], 1),
                         "newton_per_substep": st["newton_iters"] / max(st["substeps"], 1),
                         "deviation_from_cd1": dev})
    return {"sweep": "dt x C_d on the GRF 128^3 grid", "precision": args.sweep_precision, "cells": n,
            "rows": rows}


def run_sweep_z(args):
    """Metallicity and C_d sweep on the initial Bonnor-Ebert sphere (Sec. 4.3,
    the settings of its solver-performance comparison): the LI method (mixed
    batched, plain FP64 batched) and the Newton-Raphson reference on the same
    GPU; cell-updates/s, substeps per cell and the LI - NR difference."""
    import torch
    import paper_2604_21438_gb300 as sf
    rows = []
    for Z, cds in ((1.0, (1.0, 10.0, 100.0, 1e3, 1e4)), (1e-2, (1e3,)), (1e-4, (1e3,))):
        cells, off, _ = inputs.cells_be(Z)
        dt = inputs.be_dt()
        bdt = np.full(len(off) - 1, dt)
        n = len(cells["n_H"])
        d = sf.to_device(cells)
        pristine = {k: d[k].clone() for k in sf.STATE_FIELDS}
        for cd in cds:
            row = {"Z": Z, "C_d": cd * 1e4, "cells": n, "dt_yr": dt / YR}
            outs = {}
            for leg in ("mixed", "fp64", "nr"):
                kw = {"n_sub_max": 2000} if leg == "nr" else {}
                s = sf.Solver("mixed" if leg == "mixed" else "fp64", Z=Z, **kw)
                times = []
                for rep in range(4):
                    for k in sf.STATE_FIELDS:
                        d[k].copy_(pristine[k])
                    if rep == 1:
                        s.stats_reset()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    if leg == "nr":
                        s.step_nr(d, dt, cd)
                    else:
                        s.step_batched(d, off, bdt, cd)
                    b.record()
                    torch.cuda.synchronize()
                    if rep >= 1:
                        times.append(a.elapsed_time(b))
                st = s.stats()
                s.close()
                outs[leg] = sf.to_host({k: d[k] for k in sf.STATE_FIELDS + ("n_sub", "status")})
                ms = float(np.mean(times))
                row[leg] = {"cell_updates_per_s": n / (ms * 1e-3), "ms": ms,
                            "n_sub_av": st["substeps"] / max(st["cells"], 1),
                            "tight_fraction": st["tight_cells"] / max(st["cells"], 1),
                            "noconv_cells": st["noconv_cells"]}
            for name, a in (("li_vs_nr", outs["fp64"]), ("mixed_vs_fp64", outs["mixed"])):
                b = outs["nr"] if name == "li_vs_nr" else outs["fp64"]
                row[name] = {}
                for k in ("T_g", "T_d"):
                    e = np.abs(a[k] - b[k]) / np.abs(b[k])
                    row[name][k] = {"max": float(e.max()), "p99": float(np.percentile(e, 99)),
                                    "median": float(np.median(e))}
            rows.append(row)
        del d, pristine
    return {"sweep": "Z x C_d on the initial Bonnor-Ebert sphere", "rows": rows}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.sweep:
        if rank == 0:
            print(json.dumps(run_sweep(args)))
        return
    if args.sweep_z:
        if rank == 0:
            print(json.dumps(run_sweep_z(args)))
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    init_dist(world, local)
    line = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
