#!/usr/bin/env python
"""Throughput of the staggered-mesh MHD step on GB300.

Workload: compressible MHD turbulence in a periodic 512^3 box (gamma 5/3,
rho 1, P 1/gamma, B0 = 0.3 z, Gaussian random solenoidal velocity with
E(k) ~ k^-2 for 1 <= k <= 4 at rms Mach 0.5), Richtmyer-Morton shock
viscosity, energy diffusion, resistivity and quenching on, FP32 storage and
arithmetic, Courant time step computed on the device every step.  A "step" is
one full low-storage RK3 step (three right-hand-side evaluations).

Prints one JSON line.  `value` is zone-updates/s over the whole job with the
state resident in HBM, timed with per-kernel instrumentation off; `e2e`
repeats the measurement through the host-memory entry point (copies
included).  `roofline` is the step's HBM roofline: the minimal algorithmic
traffic of a full RK3 step (288 B per zone: the eight FP32 state arrays read
per stage, the time-derivative arrays read and written, the state written)
times the zone-updates/s, over the measured copy bandwidth.  `alu_roofline`
sets the oracle's operation count per zone per step against the FP32 issue
peak of the GPU (SMs x 128 lanes x 2 flops per multiply-add x the SM clock
sampled under load).  `kernels` reports each kernel's share of a step and
the bytes of the arrays it reads and writes, from a separate instrumented
pass.  `cpu_baseline` times the FP64 CPU oracle on a bounded sample of the
same workload.

--impl reference times that CPU oracle alone (the comparison arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zone-updates/s per full MHD step (FP32) at 512^3 + % HBM roofline; adjoint step cost"
UNIT = "zone-updates/s"
PHYS = dict(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=1)
STEP_BYTES_PER_ZONE = 288       # minimal HBM bytes per zone per RK3 step (8 FP32 fields, 2N storage)
CPU_SAMPLE_N = 128              # oracle sample grid (cells per axis)
CPU_SAMPLE_SECONDS = 12.0       # run oracle steps until this much host time is spent
CPU_SAMPLE_MAX_STEPS = 30
REF_N = 96                      # per-step sample grid of the reference (oracle) arm

# Distinct FP32 arrays each kernel reads + writes per launch (every array
# touched once), for the viscous, quenched workload: the traffic of the
# arrays the design materialises, not the method's algorithmic minimum.
# k_div: per stage, over its three launches (momentum; mass and energy;
# induction; their arrays are disjoint): stage 1 (Courant) reads 25 and
# writes 8; stages 2 and 3 read 38 (fluxes, state, previous dfdt) and write
# 16; k_update is the stage-1 update of all 8 fields (f, dfdt in; f out).
KERNEL_ARRAYS = {"k_lr_ed": 4, "k_vel": 10, "k_nu_raw": 9, "k_nu_max": 2, "k_nu_smooth": 3,
                 "k_nu_maxsmooth": 3,
                 "k_nu_faces": 4, "k_tau": 26, "k_edge": 28, "k_flux": 40, "k_flux_e": 17,
                 "k_div": (33 + 54 + 54) / 3.0, "k_update": 24}
# DRAM bytes (read + write) per cell per launch from one ncu capture of each
# kernel on the same workload at 192^3 (traffic grows with the cells).  Only
# kernels unchanged since their capture.
NCU_TRAFFIC_PER_CELL = {"k_flux": 1112.1e6 / 192 ** 3, "k_flux_e": 500.6e6 / 192 ** 3,
                        "k_edge": 762.6e6 / 192 ** 3, "k_tau": 710.2e6 / 192 ** 3,
                        # per unit of three launches, the mean over the three stages
                        "k_div": (940.6e6 + 2 * 1539.8e6) / 3 / 192 ** 3}
# DRAM bytes per zone of one whole step (read + write summed over its 38
# launches), from an ncu launch list with DRAM counters of the same step at
# 192^3 (traffic grows with the cells): 10.537 GB + 5.189 GB over 192^3 zones.
STEP_TRAFFIC_PER_ZONE = (10537.0e6 + 5189.3e6) / 192 ** 3
# Launches that together form one unit of KERNEL_ARRAYS.
LAUNCHES_PER_UNIT = {"k_div": 3}
FP32_LANES_PER_SM = 128         # FP32 multiply-add lanes per SM (4 partitions x 32)


def flops_per_zone(workload="turbulence"):
    """Operations per zone per RK3 step counted from the oracle's operator
    list (tests/golden/count_flops.py writes the file; this only reads it)."""
    p = os.path.join(ROOT, "tests", "golden", "flops_per_zone.json")
    return json.load(open(p))[workload]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def max_over_ranks(ms, device="cpu"):
    """The slowest rank's time: every rank's result is divided by it, so the
    job's throughput is the work of all ranks over the longest wall time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_rank, steps, ms_max, world):
    """Whole-job zone-updates/s: replicas are independent (weak scaling)."""
    return world * cells_per_rank * steps / (ms_max * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.idx = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(n=CPU_SAMPLE_N, seconds=CPU_SAMPLE_SECONDS, max_steps=CPU_SAMPLE_MAX_STEPS):
    """FP64 oracle, as it stands, on the host cores: Courant RK3 steps of the
    same physics and initial-condition recipe on an n^3 box, until `seconds`
    of host time (at least one step)."""
    import torch

    import oracle
    import workloads as inputs
    w = inputs.turbulence(n)
    g = oracle.Grid(*w.shape, *w.spacing)
    p = oracle.Params(**{k: (bool(v) if k == "do_quench" else v) for k, v in PHYS.items()})
    f = [torch.tensor(a) for a in w.fields]
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        f, _ = oracle.step(f, g, p)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    t = time.perf_counter() - t0
    return {"value": n ** 3 * steps / t, "unit": UNIT, "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": "%d Courant RK3 steps of the same physics and initial-condition recipe "
                      "on a %d^3 periodic box (FP64, whole-array torch CPU ops), %.1f s" % (steps, n, t)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import torch
    n = REF_N
    steps_per = 1
    import oracle
    import workloads as inputs
    w = inputs.turbulence(n)
    g = oracle.Grid(*w.shape, *w.spacing)
    p = oracle.Params(**{k: (bool(v) if k == "do_quench" else v) for k, v in PHYS.items()})
    f = [torch.tensor(a) for a in w.fields]
    for _ in range(args.warmup):
        f, _ = oracle.step(f, g, p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, _ = oracle.step(f, g, p)
    t = time.perf_counter() - t0
    v = n ** 3 * args.steps * steps_per / t
    sample = ("each step one Courant RK3 step of the 512^3 workload's physics and initial-"
              "condition recipe on a %d^3 box (FP64 oracle, whole-array torch CPU ops)" % n)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "MHD turbulence, %d^3 sample of the 512^3 workload" % n,
                      "grid": [n, n, n], "parallelism": "host cores"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-ot2d", action="store_true",
                    help="skip the Orszag-Tang 1024^2 x 1, 2000-step run")
    ap.add_argument("--stratified", action="store_true",
                    help="also run the stratified atmosphere with rigid z walls: 768^2 x 384 "
                         "for 200 FP32 steps, and 384^2 x 192 FP32 against the FP64 op graph")
    ap.add_argument("--stratified-size", type=int, nargs=3, default=[768, 768, 384],
                    metavar=("NX", "NY", "NZ"))
    ap.add_argument("--stratified-steps", type=int, default=200)
    ap.add_argument("--scalar-cells", action="store_true",
                    help="one cell per thread in the fused kernels (default: four x-cells)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="print only the adjoint step cost (Orszag-Tang 3D 128^3) as a JSON line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_2405_02483_gb300 as S
    import workloads as inputs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if args.adjoint_only:
        if rank == 0:
            print(json.dumps({"adjoint": adjoint_cost(S, torch)}), flush=True)
        return
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    w = inputs.turbulence(n, device="cuda")
    refs, dev = S.split_state(w.fields)
    del w
    params = S.default_params(ref=refs, scalar_cells=int(args.scalar_cells), **PHYS)
    sim = S.Sim((n, n, n), (1.0 / n,) * 3, params)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        sim.step(dev, None)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    l0 = sim.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(dev, None)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = sim.launches() - l0
    clk = clocks.stop()
    ms = max_over_ranks(ms, device="cuda")
    ms_step = ms / args.steps
    value = job_value(n ** 3, args.steps, ms, ws)

    # Per-kernel CUDA-event times, in a separate instrumented pass (events on
    # the launch stream around every launch) after the headline timing.
    sim.timing(True)
    ksteps = max(2, min(args.steps, 5))
    for _ in range(ksteps):
        sim.step(dev, None)
    ktimes = sim.kernel_times()
    sim.timing(False)

    # The step's HBM roofline (algorithmic bytes per zone per step) and its
    # FP32 ALU roofline (oracle operation count per zone per step).
    peak, peak_kind = peaks()
    step_gbs = STEP_BYTES_PER_ZONE * (value / ws) / 1e9
    roof = {"kernel": "whole RK3 step (every launch of the three stages)", "bound": "hbm",
            "achieved": step_gbs, "peak": peak, "unit": "GB/s", "frac": step_gbs / peak,
            "peak_kind": peak_kind, "bytes_per_zone": STEP_BYTES_PER_ZONE,
            "traffic": (STEP_TRAFFIC_PER_ZONE * n ** 3 if STEP_TRAFFIC_PER_ZONE else None),
            "traffic_unit": "DRAM bytes per step"}
    props = torch.cuda.get_device_properties(local)
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    alu_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    fz = flops_per_zone("turbulence")
    alu_ach = fz["flops"] * (value / ws) / 1e12
    alu = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
           "frac": alu_ach / alu_peak, "flops_per_zone": fz["flops"],
           "transcendentals_per_zone": fz["transc"],
           "peak_derivation": "%d SMs x %d FP32 lanes x 2 flops per multiply-add x %.0f MHz "
                              "(median SM clock sampled during the timed steps)"
                              % (props.multi_processor_count, FP32_LANES_PER_SM, sm_mhz),
           "ms_per_step_at_peak": fz["flops"] * n ** 3 / (alu_peak * 1e12) * 1e3,
           "hbm_ms_per_step_at_peak": STEP_BYTES_PER_ZONE * n ** 3 / (peak * 1e9) * 1e3}
    tot = sum(x[0] for x in ktimes.values()) or 1.0
    kernels = {}
    for k, v in sorted(ktimes.items(), key=lambda kv: -kv[1][0]):
        per = v[0] / v[1] * LAUNCHES_PER_UNIT.get(k, 1)
        d = {"ms_per_launch": v[0] / v[1], "launches_per_step": v[1] / ksteps,
             "share": v[0] / tot}
        if k in KERNEL_ARRAYS:
            b = KERNEL_ARRAYS[k] * 4.0 * n ** 3
            d["array_bytes_per_unit"] = b
            d["array_gbs"] = b / (per * 1e-3) / 1e9
            d["array_frac"] = d["array_gbs"] / peak
        if k in NCU_TRAFFIC_PER_CELL:
            d["ncu_dram_bytes_per_unit"] = NCU_TRAFFIC_PER_CELL[k] * n ** 3
        kernels[k] = d

    # End to end through the host-memory entry point (copies inside).
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(sim, dev, args.e2e_steps, ws, n)

    out = {"metric": METRIC
, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "MHD turbulence %d^3, RM viscosity + quench, Courant dt" % n,
                      "grid": [n, n, n], "l2": "inputs larger than L2 (state %.1f GiB)"
                      % (8 * 4 * n ** 3 / 2 ** 30),
                      "parallelism": "replicas" if ws > 1 else "single GPU"},
           "roofline": roof, "alu_roofline": alu, "kernels": kernels,
           "e2e": e2e, "gpu_launches": launches, "clocks": clk}

    if rank == 0 and not args.no_adjoint:
        out["adjoint"] = adjoint_cost(S, torch)
    if rank == 0 and not args.no_ot2d:
        out["orszag_tang_2d"] = orszag_tang_2d(S, torch)
        out["ideal_mhd"] = ideal_mhd(S, torch, peak, n=n)
    sim.close()
    del dev
    torch.cuda.empty_cache()
    if rank == 0 and args.stratified:
        out["stratified_atmosphere"] = stratified_atmosphere(S, torch, tuple(args.stratified_size),
                                                             steps=args.stratified_steps,
                                                             every=min(20, args.stratified_steps))
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def ideal_mhd(S, torch, peak, n=512, steps=5):
    """The same 512^3 turbulence state and Courant steps with every diffusion
    term off (ideal MHD, the physics of the linear-wave workload): its step
    time and both rooflines, for context beside the viscous headline."""
    import workloads as inputs
    w = inputs.turbulence(n, device="cuda")
    refs, dev = S.split_state(w.fields)
    del w
    sim = S.Sim((n, n, n), (1.0 / n,) * 3, S.default_params(ref=refs))
    for _ in range(3):
        sim.step(dev, None)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        sim.step(dev, None)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sim.close()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    alu_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2070.0e6
    zps = n ** 3 / (ms * 1e-3)
    fz = flops_per_zone("ideal")["flops"]
    return {"workload": "MHD turbulence %d^3, ideal MHD (no diffusion), Courant dt" % n,
            "ms_per_step": ms, "value": zps, "unit": UNIT,
            "hbm_frac": STEP_BYTES_PER_ZONE * zps / (peak * 1e9),
            "alu_frac": fz * zps / alu_peak, "flops_per_zone": fz}


def orszag_tang_2d(S, torch, n=1024, steps=2000, every=10):
    """The Orszag-Tang vortex (eq. initOT) at its stated size, n x n x 1, with
    the benchmark's physics for `steps` Courant steps; FP64 diagnostics every
    `every` steps.  Zone-updates/s over the steps alone (CUDA events around
    each run of `every` steps; the diagnostics between them are not timed)."""
    import workloads as inputs
    w = inputs.orszag_tang(n, n, 1)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, **PHYS))
    d0 = sim.diagnostics(dev)
    ms, log = 0.0, []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps // every):
        e0.record()
        sim.run(dev, every)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        log.append(sim.diagnostics(dev))
    sim.close()
    etot = [d[4] + d[5] + d[6] for d in [d0] + log]
    return {"workload": "Orszag-Tang %dx%dx1, RM viscosity + quench, Courant dt" % (n, n),
            "steps": steps, "value": n * n * steps / (ms * 1e-3), "unit": UNIT,
            "log_every": every, "log_entries": len(log),
            "max_rel_mass_drift": max(abs(d[0] - d0[0]) / d0[0] for d in log),
            "max_abs_net_px": max(abs(d[1]) for d in log),
            "max_abs_net_py": max(abs(d[2]) for d in log),
            "max_abs_net_pz": max(abs(d[3]) for d in log),
            "max_div_b": max(d[7] for d in log), "max_rms_div_b": max(d[8] for d in log),
            "rel_total_energy_change": (etot[-1] - etot[0]) / etot[0],
            "kinetic_first_last": [log[0][5], log[-1][5]],
            "magnetic_first_last": [log[0][6], log[-1][6]],
            "nonfinite": max(d[9] for d in log)}


def stratified_atmosphere(S, torch, size=(768, 768, 384), steps=200, every=20):
    """The isothermal atmosphere of 8 scale heights (rho = exp(-8 z), g = 8
    along -z, velocity noise 1e-3, B = (0, 0, 0.1)) in a (2, 2, 1) box with
    rigid z walls (reading R25; 14 ghost planes at each end continue the
    atmosphere) and the benchmark's physics, for `steps` Courant steps:
    (1) FP32 at `size`, zone-updates/s of the physical cells over the steps
    alone and FP64 totals every `every` steps, with rigid walls and (1b) with
    the stellar-atmosphere boundaries (readings R26, R27); (2) FP32 against the
    FP64 op graph at half the resolution with the stellar-atmosphere boundaries
    but no potential-field relaxation (the op graph does not take it),
    the same dt every step, the error of each field on the physical planes
    after the steps."""
    import numpy as np
    import workloads as inputs
    G = S.ZGHOST_MIN
    phys = dict(PHYS, zwalls=2, zghost=G)
    res = {"workload": "stratified atmosphere %dx%dx%d (+%d ghost planes each end), rigid z "
                       "walls, RM viscosity + quench, gravity 8, Courant dt" % (size + (G,)),
           "steps": steps}
    # (1) full size, FP32
    w = inputs.stratified_atmosphere(*size, zghost=G)
    refs, dev = S.split_state(w.fields)
    shape, spacing = w.shape, w.spacing
    del w
    sim = S.Sim(shape, spacing, S.default_params(ref=refs, g=(0.0, 0.0, -8.0), **phys))
    d0 = sim.diagnostics(dev)
    ms, log = 0.0, []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps // every):
        e0.record()
        sim.run(dev, every)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        log.append(sim.diagnostics(dev))
    sim.close()
    ncell = size[0] * size[1] * size[2]
    lb, ub = G, G + size[2] - 1
    umax = max(float((dev[c][lb:ub + 1].double() + refs[c]).abs().max()) for c in (1, 2, 3))
    res.update({"value": ncell * steps / (ms * 1e-3), "unit": UNIT + " (physical cells)",
                "ms_per_step": ms / steps, "cells_with_ghosts": shape[0] * shape[1] * shape[2],
                "mass_first_last": [d0[0], log[-1][0]],
                "kinetic_first_last": [d0[5], log[-1][5]],
                "max_abs_momentum_last": umax,
                "max_div_b": max(d[7] for d in log), "nonfinite": max(d[9] for d in log)})
    del dev
    torch.cuda.empty_cache()
    # (1b) the same atmosphere with the stellar-atmosphere boundaries (R26):
    # the bottom relaxes to its initial plane values on t = 0.1, the inflow
    # switch on the noise speed, the top limits at their defaults, and the
    # top's horizontal field relaxes toward the potential field on t = 2e-3,
    # about ten Courant steps (R27).
    w = inputs.stratified_atmosphere(*size, zghost=G)
    rb, Eb = float(w.fields[0][G, 0, 0]), float(w.fields[4][G, 0, 0])
    refs, dev = S.split_state(w.fields)
    shape, spacing = w.shape, w.spacing
    del w
    popen = dict(PHYS, zwalls=3, zghost=G, bdry_t=0.1, bdry_rho=rb, bdry_E=Eb, bdry_u=1e-3,
                 top_tpot=2e-3)
    sim = S.Sim(shape, spacing, S.default_params(ref=refs, g=(0.0, 0.0, -8.0), **popen))
    o0 = sim.diagnostics(dev)
    ms, olog = 0.0, []
    for _ in range(steps // every):
        e0.record()
        sim.run(dev, every)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        olog.append(sim.diagnostics(dev))
    # per-kernel CUDA-event times of two more steps (boundary kernels included)
    sim.timing(True)
    for _ in range(2):
        sim.step(dev, None)
    kt = sim.kernel_times()
    sim.timing(False)
    sim.close()
    ktot = sum(v[0] for v in kt.values()) or 1.0
    kshare = {k: {"ms_per_step": v[0] / 2, "share": v[0] / ktot}
              for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])}
    lb, ub = G, G + size[2] - 1
    umax = max(float((dev[c][lb:ub + 1].double() + refs[c]).abs().max()) for c in (1, 2, 3))
    res["open_boundaries"] = {
        "kernels": kshare,
        "value": ncell * steps / (ms * 1e-3), "unit": UNIT + " (physical cells)",
        "ms_per_step": ms / steps, "mass_first_last": [o0[0], olog[-1][0]],
        "kinetic_first_last": [o0[5], olog[-1][5]], "max_abs_momentum_last": umax,
        "max_div_b": max(d[7] for d in olog), "nonfinite": max(d[9] for d in olog)}
    del dev
    torch.cuda.empty_cache()
    # (2) half resolution, stellar-atmosphere boundaries: FP32 fused path
    # against the FP64 op graph
    half = (size[0] // 2, size[1] // 2, size[2] // 2)
    w = inputs.stratified_atmosphere(*half, zghost=G)
    rb, Eb = float(w.fields[0][G, 0, 0]), float(w.fields[4][G, 0, 0])
    refs, d32 = S.split_state(w.fields)
    d64 = [torch.tensor(a - r, dtype=torch.float64).cuda() for a, r in zip(w.fields, refs)]
    shape, spacing = w.shape, w.spacing
    del w
    popen = dict(PHYS, zwalls=3, zghost=G, bdry_t=0.1, bdry_rho=rb, bdry_E=Eb, bdry_u=1e-3)
    sim = S.Sim(shape, spacing, S.default_params(ref=refs, g=(0.0, 0.0, -8.0), **popen))
    t0 = time.perf_counter()
    for _ in range(steps):
        dt = sim.step(d32, None, want_dt=True)
        sim.step_unfused_f64(d64, dt)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    sim.close()
    lb, ub = G, G + half[2] - 1
    names = ("r", "px", "py", "pz", "E", "Bx", "By", "Bz")
    err = {}
    # natural scales: rho and E their own maxima, the momenta rho c_s (c_s = 1
    # isothermal, times the largest density), the field its largest magnitude
    rmax = float((d64[0][lb:ub + 1] + refs[0]).max())
    bmax = max(float((d64[c][lb:ub + 1] + refs[c]).abs().max()) for c in (5, 6, 7))
    for c in range(8):
        a = d32[c][lb:ub + 1].double() + refs[c]
        b = d64[c][lb:ub + 1] + refs[c]
        rng_ = float(b.max() - b.min())
        e = float((a - b).abs().max())
        scale = (float(b.abs().max()) if c in (0, 4) else rmax if c in (1, 2, 3) else bmax)
        err[names[c]] = {"err_over_range": e / rng_ if rng_ > 0 else e, "range": rng_,
                         "err_over_scale": e / scale}
    r32 = d32[0][lb:ub + 1].double() + refs[0]
    r64 = d64[0][lb:ub + 1] + refs[0]
    rel = ((r32 - r64).abs() / r64).amax(dim=(1, 2)).cpu().numpy()
    q = max(1, len(rel) // 4)
    res["fp32_vs_fp64"] = {"size": list(half), "steps": steps, "per_field": err,
                           "rho_rel_err_bottom_quarter": float(np.max(rel[:q])),
                           "rho_rel_err_top_quarter": float(np.max(rel[-q:])),
                           "wall_seconds_both_paths": t64}
    return res


def run_e2e(sim, dev, steps, ws, n):
    """Same metric through stagger_step_host: every step copies the 8 state
    arrays from pinned host memory to the device, steps, and copies them back."""
    import torch
    host = [t.cpu().pin_memory() for t in dev]
    sim.step_host(host, 1, None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.step_host(host, 1, None)
    te = time.perf_counter() - t0
    nbytes = 8 * 4 * n ** 3
    return {"value": ws * n ** 3 * steps / te, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes}


def adjoint_cost(S, torch, n=128, reps=3):
    """Adjoint step cost: the FP32 adjoint of one fixed-dt step (stage
    recompute and reverse sweep included) over one forward step, on the
    Orszag-Tang 128^3 workload with the same physics."""
    import workloads as inputs
    w = inputs.orszag_tang_3d(n)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim((n, n, n), (1.0 / n,) * 3, S.default_params(ref=refs, **PHYS))
    dt = sim.courant(dev)[0]
    lam = [torch.randn_like(t) for t in dev]
    st = [t.clone() for t in dev]
    sim.step(st, dt)
    sim.step_adjoint(dev, dt, lam)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for _ in range(reps):
        sim.step(st, dt)
    e[1].record()
    torch.cuda.nvtx.range_push("adjoint_steps")   # for a profiler's range filter
    for _ in range(reps):
        sim.step_adjoint(dev, dt, lam)
    torch.cuda.nvtx.range_pop()
    e[2].record()
    torch.cuda.synchronize()
    fwd = e[0].elapsed_time(e[1]) / reps
    adj = e[1].elapsed_time(e[2]) / reps
    sim.close()
    return {"workload": "Orszag-Tang 3D %d^3, same physics" % n, "ms_forward_step": fwd,
            "ms_adjoint_step": adj, "ratio": adj / fwd}


if __name__ == "__main__":
    main()
