#!/usr/bin/env python
"""Throughput of the CTENO / CTENOZ hot path on one GB300: Mcell-RK-stage/s.

Workload: the 2D shock tube on [0,1]x[0,0.25], 512x128 squares split into triangles with a
seeded diagonal, interior vertices jittered +-0.1h (131072 cells), Sod states, transmissive
boundaries, CFL 0.4. A step is one SSP-RK3 step (three stages of reconstruction + flux/update,
with the CFL time step), i.e. the whole hot path once; the metric counts cells x 3 stages.

The headline line is the mixed-precision path (FP32 reconstruction and flux, FP64 accumulation)
with CTENO at degree 2; `variants` gives every scheme / degree / precision combination of the
workload. L2 (129 MB) is flushed between timed steps by a 256 MB write outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload shock_tube_2d|density_wave_3d_64|blast_3d_96|batch_2d] [--profile]

The default workload is the shock tube; the others are the 3D and batched configurations, measured
with the same line format (--profile runs only warm-up + steps of the headline variant, for ncu).

Under torchrun each rank advances its own replica of the workload (the path does not shard
within a mesh: replicas only); value = cells x stages of all ranks / max over ranks of the time.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "Mcell-RK-stage/s (deg 2/3, 2D tri & 3D tet), FP32-mixed vs FP64 on one GB300"
UNIT = "Mcell-RK-stage/s"
SCHEMES = {0: "CTENO", 1: "CTENOZ"}
PRECISIONS = {0: "fp64", 1: "mixed"}


class Case:
    """A workload: meshes + initial states + the scheme it is defined with."""

    def __init__(self, name, description, meshes, states, dim, scheme, degree, cfl, variants):
        self.name, self.description = name, description
        self.meshes, self.states, self.dim = meshes, states, dim
        self.scheme, self.degree, self.cfl = scheme, degree, cfl
        self.variants = variants          # (scheme, degree) pairs timed in both precisions
        self.ncells = sum(m.ncells for m in meshes)


def make_case(name, n=0):
    import workloads as W
    if name == "shock_tube_2d":
        wl = W.shock_tube_2d(512, 128)
        return Case(name, "2D shock tube [0,1]x[0,0.25], 512x128 squares -> 131072 triangles, jitter 0.1h, "
                    "Sod states, transmissive, CFL 0.4", [wl.mesh], [wl.U0], 2, 0, 2, 0.4,
                    [(0, 2), (0, 3), (1, 2), (1, 3)])
    if name == "density_wave_3d_64":
        n = n or 64
        wl = W.density_wave_3d(n)
        return Case(name, f"3D periodic unit cube, {n}^3 cubes x 6 tetrahedra -> {wl.mesh.ncells} cells, "
                    "jitter 0.08h, density wave, CFL 0.5", [wl.mesh], [wl.U0], 3, 0, 2, 0.5, [(0, 2)])
    if name == "blast_3d_96":
        n = n or 96
        wl = W.blast_3d(n)
        return Case(name, f"3D unit cube, {n}^3 cubes x 6 tetrahedra -> {wl.mesh.ncells} cells, jitter 0.08h, "
                    "blast p=10 in r<0.2, transmissive, CFL 0.3", [wl.mesh], [wl.U0], 3, 0, 3, 0.3, [(0, 3)])
    if name == "batch_2d":
        wls = W.quadrants_batch(64, seed=0)
        return Case(name, f"64 independent triangle meshes, side log-uniform in [16,256] -> "
                    f"{sum(w.mesh.ncells for w in wls)} cells, four-quadrant Riemann states, CFL 0.4, "
                    "one launch per kernel for all meshes", [w.mesh for w in wls], [w.U0 for w in wls],
                    2, 1, 2, 0.4, [(1, 2)])
    raise ValueError(name)


HEADLINE = dict(precision=1)


def variant_name(scheme, degree, precision):
    return f"{SCHEMES[scheme]}{degree + 1}_r{degree}_{PRECISIONS[precision]}"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant-steps", type=int, default=60)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="shock_tube_2d",
                    choices=["shock_tube_2d", "density_wave_3d_64", "blast_3d_96", "batch_2d"])
    ap.add_argument("--n", type=int, default=0,
                    help="override the mesh size of a 3D workload (cubes per side), e.g. for ncu")
    ap.add_argument("--launch", default="",
                    help="R,F launch values (cteno_set_launch convention) instead of autotuning")
    ap.add_argument("--profile", action="store_true",
                    help="only run the headline variant (warm-up + steps, no timing extras): a short "
                         "command for ncu")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
# distributed helpers
# ------------------------------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job_value(world: int, cells_per_rank: int, steps: int, max_ms: float) -> float:
    """Mcell-RK-stage/s of the whole job: every rank advances its own replica of `cells_per_rank`
    cells through `steps` SSP-RK3 steps (3 stages each); the time is the maximum over ranks."""
    return world * cells_per_rank * 3 * steps / (max_ms * 1e-3) / 1e6


class Dist:
    def __init__(self, world, backend):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as td
            td.init_process_group(backend=backend)
            self.td = td

    def barrier(self):
        if self.world > 1:
            self.td.barrier()

    def max(self, x: float, device=None) -> float:
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.td.all_reduce(t, op=self.td.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.td.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def alu_peak(native):
    """FP64 / FP32 FMA throughput of this GPU, measured now (cteno_measure_alu_peak)."""
    f64, f32 = native.cteno_measure_alu_peak()
    return {"fp64_tflops": round(f64, 3), "fp32_tflops": round(f32, 2)}


def recon_kernel_name(dim, degree, scheme, launch):
    """Name of the mixed-path reconstruction kernel a launch value selects."""
    args = f"{dim},{degree},float,{SCHEMES[scheme]}"
    if launch in (4096, 4097):
        return f"recon_halo_kernel<{args},{'one-tile' if launch == 4097 else 'persistent'}> x128"
    if launch >= 3072:
        return f"recon_staged_kernel<{args},lanes> x{launch - 3072}"
    if launch >= 2048:
        return f"recon_staged_kernel<{args},cells> x{launch - 2048}"
    if launch >= 1024:
        return f"recon_lanes_kernel<{args}> x{launch - 1024}"
    if launch < 0:
        return f"recon_kernel<{args},capped> x{-launch}"
    return f"recon_kernel<{args}> x{launch}"


def ncu_traffic(variant):
    """DRAM bytes per reconstruction launch from the committed ncu capture, if the kernel source
    has not changed since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    src = open(os.path.join(ROOT, "paper_2312_17042_gb300", "csrc", "recon.cuh"), "rb").read()
    if d.get("recon_cuh_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return d.get("bytes_per_launch", {}).get(variant)


def make_solver(native, case, scheme, degree, precision, stream):
    s = native.Solver(case.meshes, case.dim, degree=degree, scheme=scheme, precision=precision,
                      stream=stream, cfl=case.cfl)
    for k, U in enumerate(case.states):
        s.set_state(U, k)
    return s


def time_steps(native, s, steps, warmup, flush, torch, kernel_times=False):
    """Per-step device time (ms) of cteno_run(1) with an L2 flush before every step."""
    for _ in range(warmup):
        flush.zero_()
        s.run(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kms = []
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        s.run(1)
        ev[k][1].record()
        if kernel_times:
            kms.append(native.cteno_last_kernel_ms(s.ctx))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, (np.array(kms) if kernel_times else None)


def run_ours(args, rank, world, local):
    import torch

    from paper_2312_17042_gb300 import build as B, native

    B.build()
    torch.cuda.set_device(local)
    dist = Dist(world, "nccl")
    stream = torch.cuda.current_stream().cuda_stream
    case = make_case(args.workload, args.n)
    ncells = case.ncells
    nv = case.dim + 2
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # headline ---------------------------------------------------------------------------------
    h = dict(scheme=case.scheme, degree=case.degree, precision=HEADLINE["precision"])
    s = make_solver(native, case, h["scheme"], h["degree"], h["precision"], stream)
    if args.launch:
        blocks = tuple(int(x) for x in args.launch.split(","))
        native.cteno_set_launch(s.ctx, *blocks)
    else:
        blocks = native.cteno_autotune(s.ctx)
    if args.profile:
        time_steps(native, s, args.steps, args.warmup, flush, torch)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.workload, "blocks": blocks, "guard": s.sync()}))
        s.close()
        dist.close()
        return
    stats = native.cteno_kernel_stats(s.ctx)
    clocks = ClockSampler(local)
    dist.barrier()
    torch.cuda.synchronize()
    # the step graph as a user runs it (no timing nodes between its kernels)
    ms, _ = time_steps(native, s, args.steps, args.warmup, flush, torch)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    guard = s.sync()
    total_ms = dist.max(sum(ms), device="cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_value(world, ncells, args.steps, total_ms)
    # per-kernel durations: a separate pass of the step graph with event-record nodes between its
    # kernels (which also serialises them)
    native.cteno_set_timing(s.ctx, True)
    _, kms = time_steps(native, s, max(10, min(args.steps, 100)), 2, flush, torch, kernel_times=True)
    recon_ms_launch = float(kms[:, 0].mean()) / 3.0
    flux_ms_launch = float(kms[:, 1].mean()) / 3.0
    peaks, peak_kind = measured_peaks()
    achieved = stats[0] / (recon_ms_launch * 1e-3) / 1e9
    hv = f"{args.workload}:" + variant_name(**h) + f":{blocks[0]}"
    roofline = {"kernel": recon_kernel_name(case.dim, h["degree"], h["scheme"], blocks[0]), "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": ncu_traffic(hv),
                "algorithmic_bytes_per_launch": stats[0], "launch_ms": round(recon_ms_launch, 5),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                "flux_kernel": {"achieved_gbs": round(stats[1] / (flux_ms_launch * 1e-3) / 1e9, 1),
                                "launch_ms": round(flux_ms_launch, 5),
                                "algorithmic_bytes_per_launch": stats[1]}}
    native.cteno_set_timing(s.ctx, False)

    # end to end through the C ABI with host buffers -------------------------------------------
    # every mesh's state in one pinned host buffer, moved by the batch-wide calls
    pinned = torch.empty(nv * ncells, dtype=torch.float64, pin_memory=True).numpy()
    outs = torch.empty(nv * ncells, dtype=torch.float64, pin_memory=True).numpy()
    native.cteno_get_state_all(s.ctx, pinned)
    n_e2e = max(5, min(args.steps, 50))
    torch.cuda.synchronize()
    t_total = 0.0
    for it in range(n_e2e + 2):
        flush.zero_()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        native.cteno_set_state_all(s.ctx, pinned)
        s.run(1)
        native.cteno_get_state_all(s.ctx, outs)
        b_.record()
        b_.synchronize()
        if it >= 2:
            t_total += a.elapsed_time(b_)
    t_total = dist.max(t_total, device="cuda")
    e2e = {"value": round(whole_job_value(world, ncells, n_e2e, t_total), 2), "unit": UNIT,
           "h2d_bytes_per_step": int(pinned.nbytes), "d2h_bytes_per_step": int(outs.nbytes), "steps": n_e2e,
           "api": "cteno_set_state_all(host) + cteno_run(1) + cteno_get_state_all(host), pinned buffers"}
    s.close()

    # variants: every timed (scheme, degree) of the workload in both precisions -------------------
    variants = {}
    alu = None
    if not args.no_variants:
        alu = alu_peak(native)
        for scheme, degree in case.variants:
            for precision in (1, 0):
                name = variant_name(scheme, degree, precision)
                sv = make_solver(native, case, scheme, degree, precision, stream)
                native.cteno_autotune(sv.ctx)
                st = native.cteno_kernel_stats(sv.ctx)
                vms, _ = time_steps(native, sv, args.variant_steps, 3, flush, torch)
                native.cteno_set_timing(sv.ctx, True)
                _, vk = time_steps(native, sv, max(5, args.variant_steps // 2), 1, flush, torch, kernel_times=True)
                tot = dist.max(sum(vms), device="cuda")
                r_ms = float(vk[:, 0].mean()) / 3
                entry = {"value": round(whole_job_value(world, ncells, args.variant_steps, tot), 2),
                         "ms_per_step": round(tot / args.variant_steps, 4),
                         "recon_ms_per_launch": round(r_ms, 5),
                         "flux_ms_per_launch": round(float(vk[:, 1].mean()) / 3, 5)}
                if precision == 1:
                    entry["recon_gbs"] = round(st[0] / (r_ms * 1e-3) / 1e9, 1)
                    entry["recon_hbm_frac"] = round(entry["recon_gbs"] / peaks["hbm_gbs"], 4)
                else:
                    tfl = st[2] / (r_ms * 1e-3) / 1e12
                    entry["recon_fp64_tflops"] = round(tfl, 3)
                    entry["recon_fp64_alu_frac"] = round(tfl / alu["fp64_tflops"], 4)
                variants[name] = entry
                sv.close()
        for scheme, degree in case.variants:
            m, f = variants[variant_name(scheme, degree, 1)], variants[variant_name(scheme, degree, 0)]
            m["speedup_vs_fp64"] = round(m["value"] / f["value"], 2)

    # CPU baseline: the oracle on the host cores ---------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_timing(case, h)

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (reconstruction, flux) + f64 (accumulation)",
        "data": "synthetic (seeded jittered simplex meshes, analytic initial data)",
        "config": {"workload": case.description, "scheme": SCHEMES[h["scheme"]], "degree": h["degree"],
                   "precision": "mixed", "cells": ncells,
                   "l2": "flushed before every timed step (256 MB write, untimed)",
                   "parallelism": f"replicas x{world}", "recon_block": blocks[0], "flux_block": blocks[1],
                   "positivity_guard_cells": int(guard)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        # per stage: one reconstruction launch and one flux/update launch, or two for the
        # face-based flux schedule (face fluxes, then the per-cell update)
        "gpu_launches": 3 * (1 + (2 if blocks[1] >= 8192 else 1)) * args.steps,
        "clocks": clk,
        "variants": variants,
        "alu_peak_measured": alu,
    }
    dist.close()
    if rank == 0:
        print(json.dumps(result))


def oracle_timing(case, h, budget_s=20.0):
    """The oracle, as it stands, on the host cores: SSP-RK3 steps of the full first mesh of the
    workload (a smaller mesh of the same construction when that mesh is large), set-up excluded."""
    import workloads as W
    from oracle import Oracle, num_threads
    mesh, U0, note = case.meshes[0], case.states[0], "the full first mesh"
    if mesh.ncells > 400000:   # 3D workloads: same construction at n = 16
        sub = W.density_wave_3d(16) if case.name.startswith("density") else W.blast_3d(16)
        mesh, U0, note = sub.mesh, sub.U0, f"the same construction at n=16 ({sub.mesh.ncells} cells)"
    t0 = time.perf_counter()
    o = Oracle(mesh, degree=h["degree"], scheme=h["scheme"], cfl=case.cfl)
    setup = time.perf_counter() - t0
    o.set_state(U0)
    steps, t = 0, 0.0
    while steps < 2 or (t < budget_s / 4 and steps < 20):
        t0 = time.perf_counter()
        o.step(0.0)
        t += time.perf_counter() - t0
        steps += 1
    return {"value": round(mesh.ncells * 3 * steps / t / 1e6, 4), "unit": UNIT, "cores": num_threads(),
            "kind": "oracle",
            "sample": f"{steps} SSP-RK3 steps of {note}, {SCHEMES[h['scheme']]} degree {h['degree']}, FP64; "
                      f"set-up ({setup:.1f} s) excluded"}


# ------------------------------------------------------------------------------------------------
# reference arm: the oracle, timed as it stands on the host cores
# ------------------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import Oracle, num_threads
    case = make_case(args.workload, args.n)
    mesh, U0 = case.meshes[0], case.states[0]
    o = Oracle(mesh, degree=case.degree, scheme=case.scheme, cfl=case.cfl)
    o.set_state(U0)
    # each step is one SSP-RK3 step of the whole (first) mesh; the number of timed steps is capped
    # so the run stays within about a minute
    t0 = time.perf_counter()
    o.step(0.0)
    per = time.perf_counter() - t0
    steps = max(1, min(args.steps, int(60.0 / max(per, 1e-3))))
    warm = min(args.warmup, 1)
    for _ in range(warm):
        o.step(0.0)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(0.0)
    t = time.perf_counter() - t0
    value = mesh.ncells * 3 * steps / t / 1e6
    sample = (f"{steps} SSP-RK3 steps (of {args.steps} requested, capped to ~1 min) of the full "
              f"{mesh.ncells}-cell mesh, {SCHEMES[case.scheme]} degree {case.degree}, FP64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": round(t / steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case.description, "scheme": SCHEMES[case.scheme], "degree": case.degree},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
