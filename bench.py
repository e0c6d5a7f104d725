#!/usr/bin/env python
"""Throughput of the coupled surfactant step (cell-updates/s) on GB300.

Default workload: 3D bubble-like transport, 256^3 unit cube, sphere R = 0.125,
prescribed Hadamard-Rybczynski Stokes flow (viscosity ratio 0.01, unit
far-field velocity), F = 1 and Gamma = 0 initially, Bi = Da = 1, Langmuir EOS
sigma0 = 1, E = 0.2, dt = 5e-5.  One step = BCG advection of f and F, the
App. C implicit source system solved to tolerance,
compensated totals, EOS and Marangoni force.  In an SFX_F32 context the
App. C system is solved by a coupled Newton defect correction (FP64
contexts: Picard + multigrid).  The phase field is built once (the interface
is static in this workload).

Arms:
  (default)          libsfx on cuda:LOCAL_RANK, one independent replica per
                     rank (weak scaling); prints one JSON line on rank 0.
  --impl reference   the FP64 CPU oracle on the host cores, each step a
                     bounded 64^3 sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "cell-updates/s of coupled surfactant step (FP32/batched vs FP64), % HBM roofline"
UNIT = "cell-updates/s"
SAMPLE_N = 64          # oracle sample: centred 64^3 block of the same grid
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth (context beside the measured peak)

# DRAM bytes (read + write) per launch of a dominant kernel from one ncu
# capture, per cell of the captured grid, with a digest of the sources the
# kernel was built from: scaled by the cell count to the timed grid, and
# withdrawn (None) as soon as those sources differ from the captured ones.
NCU_TRAFFIC = {
    ("smooth_tiled", "f32", 3): {
        "bytes_per_cell": (238.25e6 + 42.65e6) / 192 ** 3,
        "sources": ["sfx_tiled.cuh", "sfx_corr3.cuh"],
        "sha256_16": "bfcde9800814a5bc",
        "capture": "profiles/corr2_tiled_hr3d192_f32.md (192^3 with the 256^3 z-chunk of 37 "
                   "planes, one launch), scaled by the cell count",
    },
}


def ncu_traffic(kind, precision, ndim, ncell):
    """Captured DRAM bytes per launch for the timed grid, or None."""
    import hashlib
    e = NCU_TRAFFIC.get((kind, precision, ndim))
    if e is None:
        return None, None
    h = hashlib.sha256()
    for f in e["sources"]:
        with open(os.path.join(ROOT, "paper_2605_27534_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != e["sha256_16"]:
        return None, "kernel sources changed since the capture"
    return e["bytes_per_cell"] * ncell, e["capture"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sfx", choices=["sfx", "reference"])
    ap.add_argument("--workload", default="hr3d", choices=["hr3d", "batch64", "vortex512"])
    ap.add_argument("--vortex-steps", type=int, default=100,
                    help="steps of the 512^2 moving-interface vortex timed beside the line "
                         "(0: skip)")
    ap.add_argument("--precision", default="f32", choices=["f64", "f32"])
    ap.add_argument("--f64-steps", type=int, default=3,
                    help="steps of the FP64 path timed beside the FP32 line (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=30,
                    help="also time the batched workload for this many steps (0: skip)")
    ap.add_argument("--vof-steps", type=int, default=20,
                    help="steps of the 256^3 geometric VoF advection timed beside the line "
                         "(0: skip)")
    ap.add_argument("--adsorption-steps", type=int, default=1000,
                    help="steps of the 128^2 FP64 no-flow adsorption workload timed beside "
                         "the line (0: skip)")
    ap.add_argument("--kinetics-steps", type=int, default=20,
                    help="steps of the flat-interface kinetics sweep timed beside the line "
                         "(0: skip)")
    ap.add_argument("--adjoint-steps", type=int, default=200,
                    help="steps of the 256^2 adjoint workload timed beside the line (0: skip)")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--sweeps", type=int, default=3,
                    help="FP32: red-black correction sweeps per Newton iteration")
    ap.add_argument("--vortex-sweeps", type=int, default=4,
                    help="FP32: correction sweeps per Newton iteration of the 2D vortex "
                         "workload (no over-relaxation in 2D)")
    ap.add_argument("--sweep-planes", type=int, default=2, choices=[1, 2],
                    help="FP32 3D: z-planes per thread of the correction sweep "
                         "(SFX_TUNE_SWEEP_PLANES)")
    ap.add_argument("--tiled", type=int, default=1, choices=[0, 1],
                    help="FP32 3D: whole red-black sweeps as tiled launches "
                         "(SFX_TUNE_TILED_SWEEP)")
    ap.add_argument("--tiled-zchunk", type=int, default=0,
                    help="z-planes per block of the tiled sweep (SFX_TUNE_TILED_ZCHUNK; "
                         "0 = chosen from the grid)")
    ap.add_argument("--fast-resid", type=int, default=1,
                    help="FP32: Newton iterations per solve with FP32 residuals "
                         "(SFX_TUNE_F32_FAST_RESID; 0 = pair residuals only)")
    ap.add_argument("--batch-fast-resid", type=int, default=2,
                    help="batched workload: FP32 residual passes per instance and step")
    ap.add_argument("--incr-resid", type=int, default=1, choices=[0, 1],
                    help="FP32 3D tiled: incremental FP32 residuals after a small pair "
                         "residual (SFX_TUNE_F32_INCR_RESID)")
    ap.add_argument("--sor", type=int, default=1,
                    help="FP32 3D: over-relaxed red updates (SFX_TUNE_F32_SOR: 1 = omega "
                         "from the diffusion numbers, 0 = Gauss-Seidel, 1001..1999 = omega_F "
                         "in 1/1000)")
    ap.add_argument("--predict", action="store_true",
                    help="FP32: start each Newton solve from x* plus the last increment "
                         "(SFX_TUNE_PREDICT 1; no gain on the 3D workload)")
    ap.add_argument("--oracle-steps", type=int, default=3)
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def max_over_ranks(x, world, device):
    """The largest of x over all ranks (timings: the job is as slow as its
    slowest replica); x itself on a single rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def residual_schedule(a, f32):
    """The residual passes of a Newton solve, as the bench configures them."""
    if not f32:
        return "pair arithmetic"
    incr = a.incr_resid and a.tiled
    if not a.fast_resid:
        return "pair passes" + (", incremental FP32 from a small one" if incr else "")
    return ("FP32 for up to %d Newton iterations per step (while the relative residual is "
            "above 1e-3), then %s" % (
                a.fast_resid, "one pair pass, then incremental FP32 from it" if incr
                else "pair passes"))


def algorithmic_bytes(kind, grid, wbytes, sweeps=3, tiled=False):
    """Unique global bytes one launch of `kind` moves on the fine grid in
    this design (reads + writes of the state and of the solver's own work
    arrays; arrays touched by half the cells count half).  N cells, d
    dimensions, 8-byte state (double or double-float pair).
    FP64 colour sweep (k_rbgs): a (all N, as neighbours) + b, lambda (N/2
      each) + d double face arrays + write a (N/2)       = 8 (2.5 + d) N
    Advection of one field: state in/out 16 N + d velocity arrays."""
    N = grid.ncell
    d = grid.ndim
    if kind == "smooth_fine":
        if wbytes == 8:
            return 8.0 * (2.5 + d) * N
        # coupled correction colour sweep (k_corr2_32): both corrections (all
        # cells, as neighbours: 8 B), the residuals and exchange Jacobian of
        # the updated half (float4: 16 B x 1/2), the d half-precision
        # drift-face arrays of both fields (2 B each), write the updated
        # half of both corrections; the last black sweep of each iteration
        # also reads and writes the state (32 B), averaged here over the
        # 2 x sweeps - 1 colour launches (the residual pass does the first
        # red half-sweep)
        # (with the tiled sweep every colour launch is the applying one)
        return (8.0 + 8.0 + 4.0 * d + 4.0 + (32.0 if tiled else 32.0 / (2 * sweeps - 1))) * N
    if kind == "smooth_tiled":
        # k_corr2_tiled, one whole sweep: the old corrections of the colour
        # updated second (4 B: the other colour's old values are not read),
        # the float4 of both colours (16 B), the d colour-packed half drift
        # arrays (4 B each), write both corrections (8 B); the staged rings
        # (halo) are re-reads, not counted
        return (4.0 + 16.0 + 4.0 * d + 8.0) * N
    if kind in ("residual", "residual_fp32") and wbytes == 4:
        # k_resid2_32: f, F, f*, F* (pairs), phi, 2 d float faces; writes the
        # residuals and exchange Jacobian (float4) and the red half of both
        # corrections
        return (16.0 + 16.0 + 4.0 + 8.0 * d + 16.0 + 4.0) * N
    if kind == "residual_incr" and wbytes == 4:
        # k_resid32_incr: the last correction (both colours, 8 B), phi, 2 d
        # float faces, the float4 read and written, the red half of both
        # corrections; neither the state nor x*
        return (8.0 + 4.0 + 8.0 * d + 32.0 + 4.0) * N
    if kind == "advect":
        return 16.0 * N + wbytes * d * N
    return None


# FP32 operations (each add, multiply or fused multiply-add counted once) of
# the App. C pair residual at an interior 3D cell, counted from the
# formulation: per field six faces of 22 (the neighbour into the diffusion
# sum 8, its face weight 1, the upwind drift product 3 and its accumulation
# 8, the diagonal weight 2) and 32 for the centre term and the scalings;
# then 44 for the exchange, 70 for both residuals, 7 for u, v and the
# residuals' rounding, 7.5 for the red half-sweep (half the cells) and 13
# for the norms.
PAIR_RESID_OPS_3D = 2 * (6 * 22 + 32) + 44 + 70 + 7 + 7.5 + 13


def alu_peak_tops(dev, clocks):
    """FP32 operations per second of the GPU at the sampled maximum SM clock:
    SMs x 128 FP32 lanes x clock (an FMA one operation), in T/s."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    return sms * 128 * mhz * 1e6 / 1e12, sms, mhz


def method_bytes(kind, grid, s):
    """Bytes one launch of `kind` must move by the per-pass minimum of the
    method's measurement plan, independent of this design's work arrays
    (s = 4 for the FP32 form, 8 for FP64; N cells, d dimensions):
      a smoother sweep of one field reads its iterate, the right-hand side,
        the coupling field and phi and writes the iterate: 5 s N; a colour
        launch of the coupled two-field sweep does half a sweep of both
        fields: 5 s N, a tiled launch a whole sweep: 10 s N; an FP64 colour
        sweep of one field: 2.5 s N;
      a residual evaluation of one field: 5 s N (the FP32 pass evaluates
        both: 10 s N);
      advection of f and F: read both and the d face velocities, write
        both: (4 + d) s N;
      totals of f and F: 2 s N; EOS and Marangoni force: (2 + d) s N."""
    N, d = grid.ncell, grid.ndim
    if kind == "smooth_fine":
        return (5.0 if s == 4 else 2.5) * s * N
    if kind == "smooth_tiled":
        return 10.0 * s * N         # a whole sweep of both fields
    if kind in ("residual", "residual_fp32", "residual_incr"):
        return (10.0 if s == 4 else 5.0) * s * N
    if kind == "advect":
        return (4.0 + d) * s * N
    if kind == "totals":
        return 2.0 * s * N
    if kind == "forces":
        return (2.0 + d) * s * N
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "sfx_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # the timed region starts once nvidia-smi is producing samples
        t0 = time.time()
        while time.time() - t0 < 2.0:
            self.fh.flush()
            if os.path.exists(self.path) and os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx = max(mx, float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() in ("active", "0x1", "1"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def sample_block(case, n_s=SAMPLE_N):
    """Centred n_s^3 block of a 3D case: same cells, h, dt and flow."""
    n = case.grid.nx
    a = (n - n_s) // 2
    s = slice(a, a + n_s)
    s1 = slice(a, a + n_s + 1)
    g = W.Grid(W.CART3D, n_s, n_s, n_s, case.grid.h)
    return (g, np.ascontiguousarray(case.C[s, s, s]),
            np.ascontiguousarray(case.ux[s, s, s1]), np.ascontiguousarray(case.uy[s, s1, s]),
            np.ascontiguousarray(case.uz[s1, s, s]))


def oracle_rate(case, steps, tol, openmp=False):
    """The FP64 CPU oracle, as it stands, on a bounded sample: the serial
    build (one thread) or the OpenMP build (its order-independent loops on
    every host core; the Gauss-Seidel sweeps stay serial).  Returns the
    rate, the seconds, the sample grid and the threads used."""
    import oracle
    oracle.use_openmp(openmp)
    try:
        g, Cs, ux, uy, uz = sample_block(case)
        p = case.params
        _, phi, _ = oracle.phase_field_build(g, Cs, case.redist_iters, case.dtau, p.eps)
        f, F = np.zeros(g.shape), np.ones(g.shape)
        t0 = time.perf_counter()
        for _ in range(steps):
            f, F, st = oracle.surfactant_step(g, p, phi, f, F, case.dt, tol, ux, uy, uz)
            oracle.marangoni(g, p, f, phi, Cs, 1)
        dt = time.perf_counter() - t0
        return g.ncell * steps / dt, dt, g, oracle.threads()
    finally:
        oracle.use_openmp(False)


def cpu_legs(case, steps, tol):
    """cpu_baseline: the OpenMP oracle over all host cores, with the
    single-thread oracle beside it (same sample)."""
    sample = "%d step(s) on the centred %d^3 block of the %d^3 workload (same h, dt, flow)" % (
        steps, SAMPLE_N, case.grid.nx)
    r1, s1, _, _ = oracle_rate(case, steps, tol, openmp=False)
    try:
        rn, sn, _, th = oracle_rate(case, steps, tol, openmp=True)
    except (OSError, subprocess.CalledProcessError) as e:   # no OpenMP toolchain
        return {"value": r1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%s: %.1f s" % (sample, s1),
                "openmp": "unavailable: %s" % str(e).splitlines()[0]}
    return {"value": rn, "unit": UNIT, "cores": th, "kind": "oracle",
            "sample": "%s, OpenMP build, %d threads: %.1f s" % (sample, th, sn),
            "single_thread": {"value": r1, "unit": UNIT, "cores": 1, "seconds": s1}}


# ------------------------------------------------------------------ arms
def run_reference(a, case, rank):
    if rank != 0:
        return
    import oracle
    try:
        oracle.build(openmp=True)
        oracle.use_openmp(True)
    except (OSError, subprocess.CalledProcessError):
        oracle.use_openmp(False)          # no OpenMP toolchain: the serial build
    threads = oracle.threads()
    g, Cs, ux, uy, uz = sample_block(case)
    p = case.params
    _, phi, _ = oracle.phase_field_build(g, Cs, case.redist_iters, case.dtau, p.eps)
    f, F = np.zeros(g.shape), np.ones(g.shape)
    times = []
    for s in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        f, F, st = oracle.surfactant_step(g, p, phi, f, F, case.dt, a.tol, ux, uy, uz)
        oracle.marangoni(g, p, f, phi, Cs, 1)
        if s >= a.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = g.ncell * a.steps / tot
    sample = "centred %d^3 block of the %d^3 workload (same h, dt, flow), %d thread(s)%s" % (
        SAMPLE_N, case.grid.nx, threads, ", OpenMP build" if threads > 1 else "")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": case.name + " (oracle sample)", "sample": sample,
                   "tol": a.tol},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_gpu_vortex(a, rank, world, local_rank):
    """The 512^2 moving-interface vortex as the line itself (FP32 context;
    the FP64 path beside it).  The working set (~40 MB) is L2-resident, so
    no HBM roofline is claimed for it."""
    import torch
    import paper_2605_27534_gb300 as sfx
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    r32 = vortex_run(a, dev, a.steps, sfx.SFX_F32, warmup=a.warmup)
    r64 = vortex_run(a, dev, max(1, a.steps // 10), sfx.SFX_F64, warmup=1)
    racdi = vortex_run(a, dev, a.steps, sfx.SFX_F32, warmup=a.warmup, rebuild_every=10)
    r32["ms_per_step"] = max_over_ranks(r32["ms_per_step"], world, dev)
    if rank != 0:
        return
    ms = r32["ms_per_step"]
    print(json.dumps({
        "metric": METRIC, "value": job_rate(r32["cells"], world, ms), "unit": UNIT,
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "vortex512: 2D single vortex 512^2, T=4, soluble (Bi=Da=1), "
                               "geometric VoF + phase-field rebuild + coupled step + Marangoni, "
                               "tol=%g" % a.tol,
                   "cells": r32["cells"], "l2": "working set L2-resident (no HBM claim)",
                   "parallelism": "replicas%d" % world},
        "roofline": None, "cpu_baseline": None, "e2e": None, "f64_path": r64,
        "f32_acdi_rebuild_every_10": racdi,
        "kernels_one_step_ms": r32["one_step_kernel_ms"],
        "newton_iters": r32["newton_or_picard_iters"],
        "speedup_vs_f64": r64["ms_per_step"] / ms, "gpu_launches": None,
    }))


def run_reference_batch(a):
    """Reference arm of the batched workload: the oracle on a bounded sample
    (two 64x128 instances), one step of each per timed step."""
    t, cells = 0.0, 0
    for s in range(a.warmup + a.steps):
        rate, secs, desc = oracle_batch_rate(a.tol, 1)
        if s >= a.warmup:
            t += secs
            cells += rate * secs
    value = cells / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "batch64 (oracle sample)", "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_gpu(a, case, rank, world, local_rank):
    import torch
    import paper_2605_27534_gb300 as sfx

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    g, p = case.grid, case.params
    prec = sfx.SFX_F32 if a.precision == "f32" else sfx.SFX_F64
    wdt = torch.float32 if prec == sfx.SFX_F32 else torch.float64
    wbytes = 4 if prec == sfx.SFX_F32 else 8
    ctx = sfx.Context.for_grid(g, prec)
    Cd = torch.from_numpy(case.C).to(dev)
    chi = torch.empty_like(Cd)
    phi = torch.empty_like(Cd)
    ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=case.redist_iters, dtau=case.dtau,
                              eps=p.eps)
    ux, uy, uz = (torch.from_numpy(u).to(dev, wdt) for u in (case.ux, case.uy, case.uz))
    f64 = prec == sfx.SFX_F64
    zeros = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    ones = torch.ones(g.shape, dtype=torch.float64, device=dev)
    # state: double (FP64 context) or double-float pairs (FP32 context)
    f = zeros.clone() if f64 else ctx.sfx_df_pack(zeros)
    F = ones.clone() if f64 else ctx.sfx_df_pack(ones)
    Cw = Cd if f64 else Cd.to(torch.float32)
    sigma = torch.empty(g.shape, dtype=wdt, device=dev)
    force = torch.empty((3,) + g.shape, dtype=wdt, device=dev)
    opts = sfx.default_opts(tol=a.tol, max_cycles=200)
    if prec == sfx.SFX_F32:   # coupled correction sweeps per Newton iteration
        opts.nu1, opts.nu2 = a.sweeps, 0
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_REUSE_DRIFT, 1)   # the interface is static
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_PREDICT, 1 if a.predict else 0)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_SWEEP_PLANES, a.sweep_planes)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_TILED_SWEEP, a.tiled)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_TILED_ZCHUNK, a.tiled_zchunk)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, a.fast_resid)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_INCR_RESID, a.incr_resid)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_SOR, a.sor)
    stats = []

    def step():
        st = ctx.sfx_surfactant_step(p, phi, f, F, case.dt, ux, uy, uz, opts=opts)
        ctx.sfx_marangoni_force(p, f, phi, Cw, sigma, force, dm_mode=1)
        stats.append((st.picard, st.vcycles, st.res_f, st.res_F, st.mass_f, st.mass_F,
                      st.converged))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(a.warmup):
        step()
    stream = torch.cuda.current_stream()
    clk = ClockSampler(local_rank)
    ctx.sfx_profile(True)
    barrier()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ctx.sfx_profile(False)
    ms = e0.elapsed_time(e1)
    prof = ctx.sfx_profile_read()
    prof_work = ctx.sfx_profile_work()   # before the end-to-end steps below add to it
    ms_max = max_over_ranks(ms, world, dev)
    cells = g.ncell * a.steps * world
    value = job_rate(g.ncell * a.steps, world, ms_max)

    # ---- end to end through the C-ABI with host buffers (pinned)
    e2e = None
    if not a.no_e2e:
        fh = f.detach().cpu().pin_memory()
        Fh = F.detach().cpu().pin_memory()
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(a.steps):
            f.copy_(fh, non_blocking=True)
            F.copy_(Fh, non_blocking=True)
            step()
            fh.copy_(f, non_blocking=True)
            Fh.copy_(F, non_blocking=True)
        s1.record(stream)
        barrier()
        ms_e = s0.elapsed_time(s1)
        ms_e = max_over_ranks(ms_e, world, dev)
        nb = 2 * g.ncell * 8
        e2e = {"value": cells / (ms_e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb}

    if rank != 0:
        return
    # ---- roofline of the dominant kernel kind
    peaks, peak_src = measured_peaks()
    top = max(prof.items(), key=lambda kv: kv[1][1])
    kind, (nl, tot_ms, nt) = top
    roof = None
    sw = max(1, opts.nu1 + opts.nu2)
    # launches that did work: in the FP32 Newton solve every launch after
    # the converged residual pass returns at once (and a rejected predicted
    # start adds one residual pass, not counted here), so they are counted
    # from the iterations, not from the launch counter
    working = {}
    tiled = prof.get("smooth_tiled", (0, 0, 0))[0] > 0
    if prec == sfx.SFX_F32 and nt == nl:
        timed = stats[-a.steps:]
        iters = sum((k - 1 if cv else k) for k, *_, cv in timed)
        if tiled:
            # sweeps 1 .. S-1 tiled, the last black colour as a colour launch
            working["smooth_tiled"] = iters * (sw - 1)
            working["smooth_fine"] = iters
        else:
            working["smooth_fine"] = iters * (2 * sw - 1)
        # the residual passes: both kinds are launched every iteration and
        # one returns at once; the library counts those that did work
        working.update(prof_work)
    ab = algorithmic_bytes(kind, g, wbytes, sw, tiled)
    mb = method_bytes(kind, g, wbytes)
    nwork = working.get(kind, nt)
    if mb is not None and nwork > 0:
        avg_s = tot_ms * 1e-3 / nwork
        achieved = mb / avg_s / 1e9
        traffic, tsrc = ncu_traffic(kind, a.precision, g.ndim, g.ncell)
        roof = {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "traffic_source": tsrc,
                "algorithmic_bytes_per_launch": mb,
                "algorithmic_bytes_note": "the method's per-pass minimum (5 s per cell per "
                                          "field and sweep, s = %d), not this design's work "
                                          "arrays" % wbytes,
                "avg_launch_ms": avg_s * 1e3, "working_launches": nwork, "launches": nl,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src,
                "per_kernel": True}
        if ab is not None:
            roof["design_bytes_per_launch"] = ab
            roof["design_bytes_achieved"] = ab / avg_s / 1e9
            roof["design_bytes_frac"] = ab / avg_s / 1e9 / peaks["hbm_gbs"]
        if kind == "residual" and prec == sfx.SFX_F32 and g.ndim == 3:
            # the pair residual is bound by its arithmetic (ncu: 73 % issue,
            # 36 % of DRAM): its roofline is the FP32 pipe, its HBM fraction
            # kept beside it
            pk, sms, mhz = alu_peak_tops(dev, clocks)
            ops = PAIR_RESID_OPS_3D * g.ncell
            hbm = {k: roof[k] for k in ("achieved", "peak", "unit", "frac")}
            roof.update({"bound": "alu", "achieved": ops / avg_s / 1e12, "peak": pk,
                         "unit": "TFLOP/s", "frac": ops / avg_s / 1e12 / pk,
                         "algorithmic_ops_per_launch": ops,
                         "algorithmic_ops_note": "%.1f FP32 operations per cell of the pair "
                                                 "residual's formulation (an FMA one "
                                                 "operation, as in the peak)"
                                                 % PAIR_RESID_OPS_3D,
                         "peak_source": "%d SMs x 128 FP32 lanes x %.0f MHz (sampled maximum "
                                        "SM clock)" % (sms, mhz),
                         "hbm": hbm})
    launches = int(sum(v[0] for v in prof.values()))
    breakdown = {}
    step_method, step_design = 0.0, 0.0
    for k, v in prof.items():
        if not v[0]:
            continue
        e = {"launches": v[0], "ms": round(v[1], 3)}
        b = algorithmic_bytes(k, g, wbytes, sw, tiled)
        m = method_bytes(k, g, wbytes)
        nw = working.get(k, v[2])
        if k in working:
            e["working_launches"] = nw
        if k in ("totals", "forces"):
            nw_m = a.steps            # one pass per step, whatever the launch count
        else:
            nw_m = nw
        if m is not None and nw > 0:
            # the method's bytes are per pass (totals and forces: per step)
            e["method_gbs"] = round(m * nw_m / (v[1] * 1e-3) / 1e9, 1)
            e["method_frac"] = round(e["method_gbs"] / peaks["hbm_gbs"], 3)
            step_method += m * nw_m
        if b is not None and nw > 0:
            e["design_gbs"] = round(b / (v[1] * 1e-3 / nw) / 1e9, 1)
            step_design += b * nw
        breakdown[k] = e
    step_s = ms_max * 1e-3
    step_level = {
        "method_bytes_per_step": step_method / a.steps,
        "method_frac": step_method / step_s / 1e9 / peaks["hbm_gbs"],
        "design_bytes_per_step": step_design / a.steps,
        "design_frac": step_design / step_s / 1e9 / peaks["hbm_gbs"],
        "note": "bytes of every pass of the timed steps (advection, residual passes, colour "
                "sweeps that did work, totals, EOS and force) over the whole step time; "
                "method = the per-pass minimum, design = this design's arrays (the kinds "
                "without a figure, e.g. set-up and flags, count as time only)"}
    cpu = None
    if not a.no_cpu:
        cpu = cpu_legs(case, a.oracle_steps, a.tol)
    pic = [s[0] for s in stats[-a.steps:]]
    f64 = None
    if prec == sfx.SFX_F32 and a.f64_steps > 0:
        f64 = f64_path(a, case, dev, f, F, phi, ux, uy, uz)
    adj = None
    if a.adjoint_steps > 0:
        adj = adjoint_summary(a, dev)
    vortex = None
    if a.vortex_steps > 0:
        vortex = {"f32": vortex_run(a, dev, a.vortex_steps, sfx.SFX_F32),
                  "f32_acdi": vortex_run(a, dev, a.vortex_steps, sfx.SFX_F32, rebuild_every=10),
                  "f64": vortex_run(a, dev, max(1, a.vortex_steps // 10), sfx.SFX_F64)}
    batch = None
    if a.batch_steps > 0:
        batch = run_gpu_batch(a, rank, 1, local_rank, steps=a.batch_steps, summary=True)
    kin = None
    if a.kinetics_steps > 0:
        kin = kinetics_sweep_run(a, dev, a.kinetics_steps)
    ads = None
    if a.adsorption_steps > 0:
        ads = adsorption_run(a, dev, a.adsorption_steps)
    vof = None
    if a.vof_steps > 0:
        vof = vof_run(a, dev, a.vof_steps)
    if roof is not None:
        roof["frac_of_nominal"] = roof["achieved"] / NOMINAL_HBM_GBS
        roof["nominal_peak"] = NOMINAL_HBM_GBS
    # the strictest bound: only the state moves (read f, F, phi and the
    # face velocities, write f and F once per step)
    sb = (2 * 2 * wbytes * 2 + 8 + wbytes * g.ndim) if prec == sfx.SFX_F32 else (
        2 * 2 * 8 + 8 + 8 * g.ndim)
    state_gbs = sb * g.ncell / (ms_max / a.steps * 1e-3) / 1e9
    state_only = {"bytes_per_cell": sb, "achieved": state_gbs, "unit": "GB/s",
                  "frac": state_gbs / measured_peaks()[0]["hbm_gbs"],
                  "note": "read f, F, phi, u and write f, F once per step"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": a.precision, "data": "synthetic",
        "config": {"workload": "%s: 3D %d^3 HR Stokes flow, sphere R=0.125, Bi=Da=1, "
                               "dt=%g, tol=%g" % (case.name, g.nx, case.dt, a.tol),
                   "cells": g.ncell, "precision": a.precision,
                   "newton_start": "x* + last increment" if a.predict else "x*",
                   "sweeps": "tiled (whole sweep per launch, zchunk %s)" % (
                             a.tiled_zchunk or "auto")
                             if (a.tiled and prec == sfx.SFX_F32) else "one launch per colour",
                   "residuals": residual_schedule(a, prec == sfx.SFX_F32),
                   "relaxation": ("%d red-black sweeps per Newton iteration, red updates "
                                  "over-relaxed (%s)" % (a.sweeps, "omega from the Jacobi-"
                                  "radius bound" if a.sor == 1 else "omega_F = %.3f" % (
                                      a.sor / 1000.0)) if a.sor else
                                  "%d red-black Gauss-Seidel sweeps per Newton iteration" %
                                  a.sweeps) if prec == sfx.SFX_F32 else None,
                   "l2": "inputs larger than L2 (state + coefficients %.2f GB)" % (
                       g.ncell * 8 * 20 / 1e9),
                   "parallelism": "replicas%d" % world,
                   "picard_per_step": statistics.mean(pic) if pic else None},
        "roofline": roof, "step_roofline": step_level, "state_only_roofline": state_only,
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks, "kernels": breakdown,
    }
    if f64 is not None:
        line["f64_path"] = f64
        line["speedup_vs_f64"] = f64["ms_per_step"] / (ms_max / a.steps)
    if batch is not None:
        line["batch64"] = batch
    if adj is not None:
        line["adjoint2d_256"] = adj
    if vortex is not None:
        line["vortex512"] = vortex
    if kin is not None:
        line["kinetics_sweep"] = kin
    if ads is not None:
        line["adsorption2d_128"] = ads
    if vof is not None:
        line["vof3d_256"] = vof
    print(json.dumps(line))


def vof_run(a, dev, steps, warmup=3, n=256):
    """Geometric VoF advection of C on the 256^3 sphere (R = 0.125) in the
    Hadamard-Rybczynski flow, SFX_F32 context (FP32 PLIC geometry, double
    C), dt = 2e-4 (face Courant numbers up to ~0.1), direction order
    alternating.  Roofline of the whole VoF step on its per-pass bytes: the
    indicator H = [C > 1/2] (C in, H out: 16 B per cell), then per direction
    the face fluxes (C of the upwind cell, u, Q out: 8 + 4 + 8 B per face)
    and the update (Q of both faces, u, H, C in, C out: 8 + 4 + 8 + 8 + 8 B
    per cell): 16 + 3 x 56 = 184 B per cell."""
    import torch
    import paper_2605_27534_gb300 as sfx
    c = W.case_hr_3d(n=n, steps=1)
    g = c.grid
    ctx = sfx.Context.for_grid(g, sfx.SFX_F32)
    Cd = torch.from_numpy(c.C).to(dev)
    u = [torch.from_numpy(x).to(dev, torch.float32) for x in (c.ux, c.uy, c.uz)]
    dt = 2e-4
    for s_ in range(warmup):
        ctx.sfx_vof_advect(*u, dt, Cd, s_ % 2)
    m0 = float(Cd.sum().item())
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s_ in range(steps):
        ctx.sfx_vof_advect(*u, dt, Cd, s_ % 2)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    peaks, src = measured_peaks()
    ab = 184.0 * g.ncell
    return {"ms_per_step": ms, "value": g.ncell / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "cells": g.ncell, "dtype": "f32 PLIC geometry, f64 C",
            "roofline": {"bound": "hbm", "achieved": ab / (ms * 1e-3) / 1e9,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ab / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "bytes_per_step": ab, "kernels": "indicator + 3 x (flux + update)"},
            "sum_C_rel_change": float(Cd.sum().item()) / m0 - 1.0}


def adsorption_run(a, dev, steps, warmup=3):
    """The 2D planar no-flow adsorption workload in FP64 as specified: 128^2
    unit box, circle R = 0.25, phase-field width 1.5 cells, F = 1 outside and
    0 inside, clean interface, Langmuir k_a = 1, k_d = 0.1, D = 1e-2,
    multigrid to residual 1e-10, dt = 1e-3, `steps` steps (1000: t = 1)
    timed as one run (latency-bound: 16 k cells).  Reports the interface
    average Gamma = sum V f / sum V delta_phi at the end and the total."""
    import torch
    import paper_2605_27534_gb300 as sfx
    c = W.case_adsorption_2d(n=128, steps=steps, tol=1e-10)
    g, p = c.grid, c.params
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    Cd = torch.from_numpy(c.C).to(dev)
    chi, phi, delta = torch.empty_like(Cd), torch.empty_like(Cd), torch.empty_like(Cd)
    ctx.sfx_phase_field_build(Cd, chi, phi, delta, iters=c.redist_iters, dtau=c.dtau, eps=p.eps)
    F0 = torch.from_numpy(c.F0).to(dev)
    f, F = torch.zeros_like(F0), F0.clone()
    opts = sfx.default_opts(tol=1e-10, max_cycles=200)
    M0 = sum(ctx.sfx_totals([f, F]))
    for _ in range(warmup):                      # warm-up on a scratch copy
        ff, FF = f.clone(), F.clone()
        ctx.sfx_surfactant_step(p, phi, ff, FF, c.dt, opts=opts)
    pic, conv = [], True
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        st = ctx.sfx_surfactant_step(p, phi, f, F, c.dt, opts=opts)
        pic.append(st.picard)
        conv = conv and bool(st.converged)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mf, mF = ctx.sfx_totals([f, F])
    md = ctx.sfx_totals([delta])[0]
    return {"ms_total": ms, "ms_per_step": ms / steps, "value": g.ncell * steps / (ms * 1e-3),
            "unit": UNIT, "steps": steps, "cells": g.ncell, "dtype": "f64",
            "picard_per_step": statistics.mean(pic), "all_converged": conv,
            "t_end": steps * c.dt, "gamma_mean_end": mf / md,
            "mass_rel_drift": (mf + mF - M0) / M0}


def kinetics_sweep_run(a, dev, steps, n_inst=512, ny=256, nx=8, warmup=3):
    """The flat-interface kinetics of Sec. 4.3 as a batched sweep: n_inst
    planar columns (nx x ny over y in [-4, 4], interface at y = 0, F = 1 above
    a clean interface, no flow) with log10 Bi, log10 Da uniform in [-2, 2],
    stepped together in one graph per step (SFX_F32 batched form).  The
    phase field is built once on the GPU (every column has the same
    interface) and declared static."""
    import torch
    import paper_2605_27534_gb300 as sfx
    cases = W.batch_flat_kinetics(n_inst, ny, nx)
    c0 = cases[0]
    g = c0.grid
    ctx = sfx.Context.for_grid(g, sfx.SFX_F32)
    Cd = torch.from_numpy(c0.C).to(dev)
    chi, phi1 = torch.empty_like(Cd), torch.empty_like(Cd)
    ctx.sfx_phase_field_build(Cd, chi, phi1, None, iters=c0.redist_iters, dtau=c0.dtau,
                              eps=c0.params.eps)
    phi = phi1.reshape(-1).repeat(n_inst)
    B = sfx.Batch([(nx, ny, g.h, c.dt, c.params) for c in cases], geom=sfx.SFX_PLANAR2D)
    B.sfx_batch_reuse_phi(True)
    F0 = torch.from_numpy(np.concatenate([c.F0.ravel() for c in cases])).to(dev)
    f = sfx.sfx_df_pack(torch.zeros_like(F0))
    F = sfx.sfx_df_pack(F0)
    block, sweeps, budget = B.sfx_batch_autotune(phi, f, F, a.tol)
    for _ in range(warmup):
        B.sfx_batch_step(phi, f, F, a.tol)
    B.sfx_batch_work(reset=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        B.sfx_batch_step(phi, f, F, a.tol)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rp, _ = B.sfx_batch_work()
    st = B.sfx_batch_stats()
    ncell = n_inst * nx * ny
    # interface concentration Gamma = sum h^2 f / (interface length nx h)
    gam = np.array(st["mass_f"]) / (nx * g.h)
    return {"ms_per_step": ms, "value": ncell / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "instances": n_inst, "cells": ncell, "grid": "%dx%d planar, h=%g" % (nx, ny, g.h),
            "dt": c0.dt, "schedule": {"block": block, "sweeps": sweeps, "iteration_budget": budget},
            "newton_iters_mean": float(np.mean(np.array(rp) / steps)),
            "all_converged": bool(all(st["converged"])),
            "gamma_range_after": [float(gam.min()), float(gam.max())],
            "t_after": c0.dt * (warmup + steps)}


def vortex_run(a, dev, steps, prec, warmup=3, rebuild_every=1):
    """The 2D moving-interface workload: 512^2 single vortex (T = 4) with
    the soluble surfactant (Bi = Da = 1), from t = 0.  One step = geometric
    VoF advection of C, the phase field (rebuilt from C, or with
    rebuild_every > 1 carried by one ACDI step with zeta = 1.1 max|u| and
    rebuilt from C every rebuild_every steps), the coupled step with the
    same velocity, EOS and Marangoni force.  The face velocities are
    cos(pi t/T) times the t = 0 field (the stream function factorises),
    scaled on the device before each step (input preparation)."""
    import torch
    import paper_2605_27534_gb300 as sfx
    c = W.case_vortex_2d(n=512, soluble=True)
    g, p = c.grid, c.params
    T = c.extra["T"]
    f32 = prec == sfx.SFX_F32
    vt = torch.float32 if f32 else torch.float64
    ctx = sfx.Context.for_grid(g, prec)
    if f32:   # the phase field is rebuilt every step: FP32 redistancing (fused 2D kernel)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_REDIST, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_SOR, a.sor)
    u0h = W.single_vortex_faces(512, g.h, 0.0, T)
    umax0 = max(float(np.abs(x).max()) for x in u0h)
    u0 = [torch.from_numpy(x).to(dev, vt) for x in u0h]
    u = [torch.empty_like(x) for x in u0]
    Cd = torch.from_numpy(c.C).to(dev)
    chi, phi, delta = torch.empty_like(Cd), torch.empty_like(Cd), torch.empty_like(Cd)
    ctx.sfx_phase_field_build(Cd, chi, phi, delta, iters=c.redist_iters, dtau=c.dtau, eps=p.eps)
    F = torch.from_numpy(c.F0).to(dev)
    f = torch.zeros_like(F)
    if f32:
        f, F = ctx.sfx_df_pack(f), ctx.sfx_df_pack(F)
    Cw = Cd.to(vt)
    sig = torch.empty(g.shape, dtype=vt, device=dev)
    force = torch.empty((2,) + g.shape, dtype=vt, device=dev)
    opts = sfx.default_opts(tol=a.tol, max_cycles=200)
    if f32:
        opts.nu1, opts.nu2 = a.vortex_sweeps, 0
    pic = []

    def step(n):
        t = (n + 0.5) * c.dt
        for x, x0 in zip(u, u0):
            torch.mul(x0, math.cos(math.pi * t / T), out=x)
        ctx.sfx_vof_advect(u[0], u[1], None, c.dt, Cd, n % 2)
        if rebuild_every <= 1 or n % rebuild_every == 0:
            ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=c.redist_iters, dtau=c.dtau,
                                      eps=p.eps)
        else:
            zeta = 1.1 * umax0 * abs(math.cos(math.pi * t / T))
            ctx.sfx_acdi_step(phi, c.dt, zeta, p.eps, u[0], u[1], clip=True)
        st = ctx.sfx_surfactant_step(p, phi, f, F, c.dt, u[0], u[1], None, opts=opts)
        if f32:
            Cw.copy_(Cd)
        ctx.sfx_marangoni_force(p, f, phi, Cw if f32 else Cd, sig, force, dm_mode=1)
        pic.append(st.picard)

    for n in range(warmup):
        step(n)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for n in range(warmup, warmup + steps):
        step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # where the time goes: one more step with the library's event brackets
    ctx.sfx_profile(True)
    step(warmup + steps)
    torch.cuda.synchronize()
    ctx.sfx_profile(False)
    kinds = {k: round(v[1], 4) for k, v in ctx.sfx_profile_read().items() if v[0]}
    return {"ms_per_step": ms, "value": g.ncell / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "cells": g.ncell, "newton_or_picard_iters": statistics.mean(pic[-steps:]),
            "dt": c.dt, "dtype": "f32" if f32 else "f64", "one_step_kernel_ms": kinds,
            "phase_field": ("rebuilt from C every step" if rebuild_every <= 1 else
                            "ACDI step, rebuilt from C every %d steps" % rebuild_every),
            "mass_C": float(Cd.sum().item()) * g.h * g.h}


def adjoint_summary(a, dev):
    """Forward and backward of the differentiable rollout on the 2D adjoint
    workload (256^2 no-flow adsorption, seeded Gamma0 perturbation, loss
    sum V |F_Ma|^2, checkpoints every 20 steps), FP32 forward."""
    import torch
    import paper_2605_27534_gb300 as sfx
    c = W.case_adjoint_2d(n=256)
    g, p = c.grid, c.params
    out = {}
    for name, prec, tol in (("f32_forward", sfx.SFX_F32, 1e-12), ("f64_forward", sfx.SFX_F64, 1e-12)):
        ctx = sfx.Context.for_grid(g, prec)
        Cd = torch.from_numpy(c.C).to(dev)
        chi, phi = torch.empty_like(Cd), torch.empty_like(Cd)
        ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=c.redist_iters, dtau=c.dtau, eps=p.eps)
        setup = sfx.RolloutSetup(context=ctx, params=p, phi=phi, C=Cd,
                                 F0=torch.from_numpy(c.F0).to(dev), dt=c.dt,
                                 nsteps=a.adjoint_steps, K=20, tol=tol)
        theta = torch.tensor([p.ka, p.kd, p.Df, p.DF], dtype=torch.float64, requires_grad=True)
        g0 = torch.from_numpy(c.gamma0).to(dev).requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = sfx.SurfactantRollout.apply(g0, theta, setup)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out[name] = {"loss": L.item(), "forward_ms": 1e3 * (t1 - t0),
                     "backward_ms": 1e3 * (t2 - t1),
                     "forward_cell_updates_per_s": g.ncell * a.adjoint_steps / (t1 - t0),
                     "dL_dtheta": [float(x) for x in theta.grad]}
    out["steps"] = a.adjoint_steps
    out["cells"] = g.ncell
    return out


def f64_path(a, case, dev, f32_f, f32_F, f32_phi, ux, uy, uz):
    """The plain FP64 GPU path on the same workload: ms per step, and the
    FP32 path's deviation from it after two steps from the same state."""
    import torch
    import paper_2605_27534_gb300 as sfx
    g, p = case.grid, case.params
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    Cd = torch.from_numpy(case.C).to(dev)
    chi = torch.empty_like(Cd)
    phi = torch.empty(g.shape, dtype=torch.float64, device=dev)
    ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=case.redist_iters, dtau=case.dtau,
                              eps=p.eps)
    u64 = [t.to(torch.float64) for t in (ux, uy, uz)]
    f = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    F = torch.ones(g.shape, dtype=torch.float64, device=dev)
    opts = sfx.default_opts(tol=a.tol, max_cycles=200)
    pic = []
    ctx.sfx_surfactant_step(p, phi, f, F, case.dt, *u64, opts=opts)   # warm-up
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.f64_steps):
        pic.append(ctx.sfx_surfactant_step(p, phi, f, F, case.dt, *u64, opts=opts).picard)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.f64_steps
    # accuracy of the FP32 path against this one: two steps from f = 0, F = 1,
    # from this path's phi (the step alone) and from the FP32 context's own
    # phi (the FP32 phase-field build as well)
    ctx32 = sfx.Context.for_grid(g, sfx.SFX_F32)
    zeros = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    f.zero_()
    F.fill_(1.0)
    o32 = sfx.default_opts(tol=a.tol, max_cycles=200, nu1=3, nu2=0)
    for _ in range(2):
        ctx.sfx_surfactant_step(p, phi, f, F, case.dt, *u64, opts=opts)
    scale = float(torch.maximum(f.abs().max(), F.abs().max()))
    errs = []
    for phi32 in (phi, f32_phi):
        f32_f.copy_(sfx.sfx_df_pack(zeros))
        f32_F.copy_(sfx.sfx_df_pack(zeros + 1.0))
        for _ in range(2):
            ctx32.sfx_surfactant_step(p, phi32, f32_f, f32_F, case.dt, ux, uy, uz, opts=o32)
        fd, Fd = sfx.sfx_df_unpack(f32_f), sfx.sfx_df_unpack(f32_F)
        errs.append(float(torch.maximum((fd - f).abs().max(), (Fd - F).abs().max())) / scale)
    return {"ms_per_step": ms, "value": g.ncell / (ms * 1e-3), "unit": UNIT, "steps": a.f64_steps,
            "picard_per_step": statistics.mean(pic), "dtype": "f64",
            "f32_rel_err_after_2_steps": errs[0],
            "f32_with_own_phi_rel_err_after_2_steps": errs[1],
            "phi_f32_build_max_abs_diff": float((f32_phi - phi).abs().max())}


# ------------------------------------------------------------------ batched
BATCH_N, BATCH_SEED = 64, 3


def batch_bytes(sizes, rp, sg, steps, sweeps, static_phi=True):
    """Algorithmic bytes of `steps` batched steps (d = 2, pairs 8 B, double
    phi 8 B, its folded copy, velocities and faces 4 B).  Per instance of N
    cells and per step: folded copy of phi (12 N), drift faces (phi 8 +
    2 fields x 2 faces x (4 + 2) = 32 N), advection of both fields (pairs in and
    out 32 N, 2 velocity arrays 8 N), copy into the iterate (32 N), totals
    (16 N) (the folded phi and the drifts are left out when phi is static:
    they are built once, outside the step); per residual pass (16 + 16 + 4 + 16 + 16 + 8 + 4 = 80 N, the
    last term the red half of both corrections); per sweep group
    2 x sweeps - 1 colour launches of (8 + 12 + 8 + 4 = 32 N, half-precision
    faces) and the state update (32 N)."""
    tot = 0.0
    for (nr, nz), r, w in zip(sizes, rp, sg):
        N = nr * nz
        per_step = (0.0 if static_phi else 12.0 + 32.0) + 40.0 + 32.0 + 16.0
        tot += N * (steps * per_step + r * 80.0 + w * ((2 * sweeps - 1) * 32.0 + 32.0))
    return tot


def batch_inputs(dev):
    """The 64 seeded instances: grids from {64x128, 128x256, 256x512},
    log-uniform Bi, Da in [1e-2, 1e2], Pe = 100, HR Stokes flow, sphere
    R = 0.2 on the axis.  Phase field built on the GPU per grid size."""
    import torch
    import paper_2605_27534_gb300 as sfx
    spec = W.batch_axi(BATCH_N, seed=BATCH_SEED)
    per_size = {}
    inst = []
    for nr, nz, Bi, Da in spec:
        c = W.case_axi(nr, nz, Bi, Da)
        if (nr, nz) not in per_size:
            ctx = sfx.Context.for_grid(c.grid, sfx.SFX_F32)
            Cd = torch.from_numpy(c.C).to(dev)
            chi = torch.empty_like(Cd)
            phi = torch.empty_like(Cd)
            ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=c.redist_iters, dtau=c.dtau,
                                      eps=c.params.eps)
            per_size[(nr, nz)] = (phi.reshape(-1), torch.from_numpy(c.ux).to(dev, torch.float32)
                                  .reshape(-1), torch.from_numpy(c.uy).to(dev, torch.float32)
                                  .reshape(-1))
        inst.append((nr, nz, c.grid.h, c.dt, c.params))
    phi = torch.cat([per_size[(i[0], i[1])][0] for i in inst])
    ur = torch.cat([per_size[(i[0], i[1])][1] for i in inst])
    uz = torch.cat([per_size[(i[0], i[1])][2] for i in inst])
    return spec, inst, phi, ur, uz


def run_gpu_batch(a, rank, world, local_rank, steps=None, summary=False):
    import torch
    import paper_2605_27534_gb300 as sfx
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    steps = steps or a.steps
    spec, inst, phi, ur, uz = batch_inputs(dev)
    sizes = [(i[0], i[1]) for i in inst]
    ncell = sum(nr * nz for nr, nz in sizes)
    B = sfx.Batch(inst)
    B.sfx_batch_reuse_phi(True)        # the interfaces are static
    B.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, a.batch_fast_resid)
    B.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_SOR, a.sor)
    ones = torch.ones(ncell, dtype=torch.float64, device=dev)
    f = sfx.sfx_df_pack(torch.zeros_like(ones))
    F = sfx.sfx_df_pack(ones)
    block, sweeps, budget = B.sfx_batch_autotune(phi, f, F, a.tol, ur=ur, uz=uz)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(a.warmup):
        B.sfx_batch_step(phi, f, F, a.tol, ur=ur, uz=uz)
    B.sfx_batch_work(reset=True)
    clk = ClockSampler(local_rank) if not summary else None
    barrier()
    if clk:
        clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        B.sfx_batch_step(phi, f, F, a.tol, ur=ur, uz=uz)
    e1.record(stream)
    barrier()
    clocks = clk.stop() if clk else None
    ms = e0.elapsed_time(e1)
    rp, sg = B.sfx_batch_work()
    st = B.sfx_batch_stats()
    ms_max = ms
    ms_max = max_over_ranks(ms, world, dev)
    value = ncell * steps * world / (ms_max * 1e-3)
    peaks, peak_src = measured_peaks()
    ab = batch_bytes(sizes, rp, sg, steps, sweeps)
    achieved = ab / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "batched step graph (all kernels of the step)",
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None,
            "algorithmic_bytes_per_step": ab / steps, "avg_step_ms": ms / steps,
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src}
    iters_mean = float(np.mean(np.array(rp) / steps))
    conv = all(st["converged"])
    sched = {"block": block, "sweeps": sweeps, "iteration_budget": budget,
             "fp32_residual_passes": a.batch_fast_resid, "sor": a.sor}
    # init, advect, copy (phi static: no fold or drifts); then, as long as
    # an instance is active, per iteration the residual, the flags, the
    # 2 sweeps - 1 colour sweeps and the loop test; totals and final
    launches_per_step = 3 + max(st["iters"]) * (2 + 2 * sweeps) + 2
    if summary:
        return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
                "cells": ncell, "instances": len(inst), "roofline_frac": roof["frac"],
                "schedule": sched, "newton_iters_mean": iters_mean, "all_converged": conv}
    e2e = None
    if not a.no_e2e:
        fh = f.detach().cpu().pin_memory()
        Fh = F.detach().cpu().pin_memory()
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(steps):
            f.copy_(fh, non_blocking=True)
            F.copy_(Fh, non_blocking=True)
            B.sfx_batch_step(phi, f, F, a.tol, ur=ur, uz=uz)
            fh.copy_(f, non_blocking=True)
            Fh.copy_(F, non_blocking=True)
        s1.record(stream)
        barrier()
        ms_e = s0.elapsed_time(s1)
        nb = 2 * ncell * 8
        e2e = {"value": ncell * steps * world / (ms_e * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}
    if rank != 0:
        return None
    cpu = None
    if not a.no_cpu:
        rate, secs, desc = oracle_batch_rate(a.tol, a.oracle_steps)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%s: %.1f s" % (desc, secs)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": a.warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch64: %d axisymmetric instances, grids from {64x128, "
                               "128x256, 256x512}, Bi and Da log-uniform in [1e-2, 1e2], "
                               "Pe=100, HR Stokes flow, seed %d, tol=%g" % (
                                   len(inst), BATCH_SEED, a.tol),
                   "cells": ncell, "precision": "f32",
                   "l2": "inputs larger than L2 (state + coefficients %.2f GB)" % (
                       ncell * 8 * 12 / 1e9),
                   "parallelism": "replicas%d" % world, "schedule": sched,
                   "newton_iters_mean": iters_mean, "all_converged": conv},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_step * steps, "clocks": clocks,
    }
    print(json.dumps(line))
    return line


def oracle_batch_rate(tol, steps):
    """The FP64 oracle, as it stands, on two 64x128 instances of the batch."""
    import oracle
    spec = [s for s in W.batch_axi(BATCH_N, seed=BATCH_SEED) if s[0] == 64][:2]
    cells, t = 0, 0.0
    for nr, nz, Bi, Da in spec:
        c = W.case_axi(nr, nz, Bi, Da)
        _, phi, _ = oracle.phase_field_build(c.grid, c.C, c.redist_iters, c.dtau, c.params.eps)
        f, F = np.zeros(c.grid.shape), np.ones(c.grid.shape)
        t0 = time.perf_counter()
        for _ in range(steps):
            f, F, _ = oracle.surfactant_step(c.grid, c.params, phi, f, F, c.dt, tol, c.ux, c.uy,
                                             None)
        t += time.perf_counter() - t0
        cells += c.grid.ncell * steps
    return cells / t, t, "%d step(s) of %d 64x128 instances of the batch, 1 thread" % (
        steps, len(spec))


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    case = W.case_hr_3d(n=a.n, steps=a.steps, tol=a.tol)
    if a.impl == "reference":
        if world > 1 and rank != 0:
            return
        if a.workload == "batch64":
            run_reference_batch(a)
        else:
            run_reference(a, case, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if a.workload == "batch64":
        run_gpu_batch(a, rank, world, local_rank)
    elif a.workload == "vortex512":
        run_gpu_vortex(a, rank, world, local_rank)
    else:
        run_gpu(a, case, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
