#!/usr/bin/env python
"""Throughput of the CTENO / CTENOZ hot path on one GB300: Mcell-RK-stage/s.

Headline workload: the 3D blast on the unit cube, 96^3 cubes split into 6 tetrahedra each
(5308416 cells), vertices jittered +-0.08h, rho = 1, u = 0, p = 10 inside r < 0.2 and 0.1
outside, transmissive boundaries, CFL 0.3, CTENO at degree 3 (20-coefficient cubic), mixed
precision (FP32 reconstruction and flux on FP64-accurate differences, FP64 accumulation and
update): the largest configuration that runs on one GPU. A step is one SSP-RK3 step (three
stages of reconstruction + flux/update, with the CFL time step), i.e. the whole hot path once;
the metric counts cells x 3 stages.

`variants` times the other configurations with the same line fields, each with its own roofline
object: the blast in FP64; the 2D shock tube (512x128 squares -> 131072 triangles, Sod, CFL 0.4)
with CTENO and CTENOZ at degree 2 and 3; the 3D density wave (64^3 x 6 tetrahedra, CTENO degree
2); the batch of 64 four-quadrant Riemann problems (1.74M triangles, CTENOZ degree 2, one launch
per kernel for all meshes); the single-material triple point (Sec. 3.4: 215000 triangles, walls,
lambda_1' = 1e4) with CWENO, TENO, CTENO and CTENOZ at fifth and seventh order, whose times per
step relative to CWENO of the same order are the GPU counterpart of the paper's Table 5; the shock
tube again with the characteristic-variable reconstruction (its cost against the conserved one); the
double Mach reflection on the paper's timing mesh size (Sec. 3.3: 715208 triangles against 714138)
with CWENO, TENO, CTENO and CTENOZ at fifth order (Table 4's comparison) and CTENO / CTENOZ at
seventh -- each in both precisions. L2 (129 MB) is flushed between timed steps by a 256 MB write outside the
timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload blast_3d_96|shock_tube_2d|density_wave_3d_64|batch_2d|triple_point_2d|
                              shock_tube_2d_characteristic|dmr_2d]
                  [--variants all|workload|none] [--profile]

--profile runs only warm-up + steps of the headline (a short command for ncu).

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
SCHEMES = {0: "CTENO", 1: "CTENOZ", 2: "CWENO", 3: "TENO"}
PRECISIONS = {0: "fp64", 1: "mixed"}
WORKLOADS = ["blast_3d_96", "shock_tube_2d", "density_wave_3d_64", "batch_2d", "triple_point_2d",
             "shock_tube_2d_characteristic", "dmr_2d"]


class Case:
    """A workload: meshes + initial states + the scheme it is defined with."""

    def __init__(self, name, description, meshes, states, dim, scheme, degree, cfl, variants, sample_centre,
                 extra=None):
        self.name, self.description = name, description
        self.extra = extra or {}          # further solver parameters (boundary kind, lambda_1')
        self.meshes, self.states, self.dim = meshes, states, dim
        self.scheme, self.degree, self.cfl = scheme, degree, cfl
        self.variants = variants          # (scheme, degree) pairs timed in both precisions
        self.ncells = sum(m.ncells for m in meshes)
        self.sample_centre = sample_centre  # centre of the oracle's sub-box sample (first mesh)


def make_case(name, n=0):
    import workloads as W
    if name == "shock_tube_2d":
        wl = W.shock_tube_2d(512, 128)
        return Case(name, "2D shock tube [0,1]x[0,0.25], 512x128 squares -> 131072 triangles, jitter 0.1h, "
                    "Sod states, transmissive, CFL 0.4", [wl.mesh], [wl.U0], 2, 0, 2, 0.4,
                    [(0, 2), (0, 3), (1, 2), (1, 3), (2, 2), (2, 3), (3, 2), (3, 3),
                     (0, 4), (1, 4), (0, 5), (1, 5), (0, 6), (1, 6)], (0.5, 0.125))
    if name == "density_wave_3d_64":
        n = n or 64
        wl = W.density_wave_3d(n)
        return Case(name, f"3D periodic unit cube, {n}^3 cubes x 6 tetrahedra -> {wl.mesh.ncells} cells, "
                    "jitter 0.08h, density wave, CFL 0.5", [wl.mesh], [wl.U0], 3, 0, 2, 0.5, [(0, 2)],
                    (0.5, 0.5, 0.5))
    if name == "blast_3d_96":
        n = n or 96
        wl = W.blast_3d(n)
        return Case(name, f"3D unit cube, {n}^3 cubes x 6 tetrahedra -> {wl.mesh.ncells} cells, jitter 0.08h, "
                    "blast p=10 in r<0.2, transmissive, CFL 0.3", [wl.mesh], [wl.U0], 3, 0, 3, 0.3, [(0, 3)],
                    (0.7, 0.5, 0.5))
    if name == "batch_2d":
        wls = W.quadrants_batch(64, seed=0)
        return Case(name, f"64 independent triangle meshes, side log-uniform in [16,256] -> "
                    f"{sum(w.mesh.ncells for w in wls)} cells, four-quadrant Riemann states, CFL 0.4, "
                    "one launch per kernel for all meshes", [w.mesh for w in wls], [w.U0 for w in wls],
                    2, 1, 2, 0.4, [(1, 2)], (0.5, 0.5))
    if name == "shock_tube_2d_characteristic":
        wl = W.shock_tube_2d(512, 128)
        return Case(name, "the 2D shock tube (131072 triangles, Sod, CFL 0.4) reconstructed in characteristic "
                    "variables (per face, Sec. 2.2 / 3.2)", [wl.mesh], [wl.U0], 2, 0, 2, 0.4,
                    [(0, 2), (0, 3), (1, 2), (1, 3)], (0.5, 0.125), extra=dict(characteristic=1))
    if name == "dmr_2d":
        wl = W.dmr_2d(n or 299)
        regions, states = W.dmr_boundary()
        return Case(name, f"double Mach reflection (Sec. 3.3), [0,4]x[0,1], {4 * (n or 299)}x{n or 299} squares -> "
                    f"{wl.mesh.ncells} triangles (the paper's timing mesh: 714138), inflow / wall / moving-shock / "
                    "transmissive boundaries, lambda_1' = 1e15, CFL 0.4", [wl.mesh], [wl.U0], 2, 0, 4, 0.4,
                    [(2, 4), (3, 4), (0, 4), (1, 4), (2, 6), (3, 6), (0, 6), (1, 6)], (0.5, 0.25),
                    extra=dict(lambda1p=1e15, regions=regions, states=states))
    if name == "triple_point_2d":
        wl = W.triple_point_2d()
        return Case(name, f"single-material triple point (Sec. 3.4), [0,7]x[0,3], 500x215 squares -> "
                    f"{wl.mesh.ncells} triangles, walls all round, lambda_1' = 1e4, CFL 0.4",
                    [wl.mesh], [wl.U0], 2, 1, 4, 0.4,
                    [(2, 4), (3, 4), (0, 4), (1, 4), (2, 6), (3, 6), (0, 6), (1, 6)], (3.5, 1.5),
                    extra=dict(lambda1p=1e4, boundary=1))
    raise ValueError(name)


def variant_name(scheme, degree, precision):
    return f"{SCHEMES[scheme]}{degree + 1}_r{degree}_{PRECISIONS[precision]}"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant-seconds", type=float, default=1.0,
                    help="timed work per variant (steps chosen from the warm-up's step time)")
    ap.add_argument("--variants", choices=["all", "workload", "none"], default="all",
                    help="all: every workload's variants; workload: the chosen workload's only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="blast_3d_96", choices=WORKLOADS)
    ap.add_argument("--n", type=int, default=0,
                    help="override the mesh size of a 3D workload (cubes per side), e.g. for ncu")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="precision of the headline (1 = mixed, 0 = FP64)")
    ap.add_argument("--launch", default="",
                    help="R,F launch values (cteno_set_launch convention) instead of autotuning")
    ap.add_argument("--profile", action="store_true",
                    help="only run the headline (warm-up + steps, no timing extras): a short command for ncu")
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


def recon_kernel_name(dim, degree, scheme, precision, launch):
    """Name of the reconstruction kernel a launch value selects."""
    args = f"{dim},{degree},{'float' if precision else 'double'},{SCHEMES[scheme]}"
    if degree >= 4 and launch >= 1536:
        return f"recon_high_kernel_occ<{degree},{SCHEMES[scheme]}> (64 registers) x{launch - 1536}"
    if degree >= 4:
        return f"recon_high_kernel<{degree},{'float' if precision else 'double'},{SCHEMES[scheme]}> x{launch - 1024}"
    if 7168 < launch <= 7176 or 7200 < launch <= 7208:
        return f"recon_pair_kernel<{args},{2 if launch < 7200 else 3} stages> x{32 * (launch % 32)}"
    if 6144 < launch <= 6152:
        return f"recon_stream_cells_kernel<{args}> x{32 * (launch - 6144)}"
    if 5120 < launch <= 5136:
        return f"recon_stream_kernel<{args},3 stages> x{32 * (launch - 5120)}"
    if 5152 < launch <= 5168:
        return f"recon_stream_kernel<{args},2 stages> x{32 * (launch - 5152)}"
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


def ncu_traffic(key):
    """DRAM bytes per reconstruction launch from the committed ncu capture, if the kernel source
    has not changed since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))

    def same(name, field):
        src = open(os.path.join(ROOT, "paper_2312_17042_gb300", "csrc", name), "rb").read()
        return d.get(field) == hashlib.sha256(src).hexdigest()

    if not same("recon.cuh", "recon_cuh_sha256"):
        return None
    degree = int(key.split(":")[1].split("_r")[1].split("_")[0])
    if degree >= 4 and not same("recon_high.cuh", "recon_high_cuh_sha256"):  # the degree 4-6 kernels
        return None
    return d.get("bytes_per_launch", {}).get(key)


def make_solver(native, case, scheme, degree, precision, stream):
    s = native.Solver(case.meshes, case.dim, degree=degree, scheme=scheme, precision=precision,
                      stream=stream, cfl=case.cfl, **case.extra)
    native.cteno_set_state_all(s.ctx, case.states)
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


def roofline_of(case, scheme, degree, precision, launch, stats, recon_ms, peaks, peak_kind, alu):
    """Roofline object of the reconstruction kernel (the dominant kernel of every workload): the
    mixed path against the measured HBM copy bandwidth, the FP64 path against the measured FP64
    FMA rate (it is bound by the FP64 pipe), both from algorithmic bytes / FLOPs per launch over
    the mean launch time measured with CUDA events inside the replayed step graph."""
    name = recon_kernel_name(case.dim, degree, scheme, precision, launch)
    gbs = stats[0] / (recon_ms * 1e-3) / 1e9
    key = f"{case.name}:{variant_name(scheme, degree, precision)}:{launch}"
    if precision == 1 or alu is None:
        return {"kernel": name, "bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": ncu_traffic(key),
                "algorithmic_bytes_per_launch": stats[0], "launch_ms": round(recon_ms, 5),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind}, of measured)"}
    tfl = stats[2] / (recon_ms * 1e-3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": round(tfl, 4), "peak": alu["fp64_tflops"],
            "unit": "TFLOP/s (FP64 FMA)", "frac": round(tfl / alu["fp64_tflops"], 4), "traffic": ncu_traffic(key),
            "algorithmic_flops_per_launch": stats[2], "launch_ms": round(recon_ms, 5),
            "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / peaks["hbm_gbs"], 4),
            "peak_source": "FP64 FMA rate measured on this GPU by cteno_measure_alu_peak (nominal 1.25 TFLOP/s)"}


def measure(native, case, scheme, degree, precision, stream, flush, torch, dist, world, steps, warmup,
            peaks, peak_kind, alu, launch=None, clocks=False, e2e=False, seconds=None):
    """One (workload, scheme, degree, precision) measurement: set-up, autotune (or the given
    launch), warm-up, the timed steps, a kernel-timing pass; optionally the clock record and the
    end-to-end number through the C ABI with host buffers."""
    s = make_solver(native, case, scheme, degree, precision, stream)
    if launch is None:
        launch = native.cteno_autotune(s.ctx)
    else:
        native.cteno_set_launch(s.ctx, *launch)
    native.cteno_set_state_all(s.ctx, case.states)
    stats = native.cteno_kernel_stats(s.ctx)
    if seconds is not None:   # variants: choose the step count from one warm-up step's time
        flush.zero_()
        t0 = time.perf_counter()
        s.run(1)
        torch.cuda.synchronize()
        one = time.perf_counter() - t0
        steps = int(max(5, min(200, seconds / max(one, 1e-6))))
    sampler = ClockSampler(torch.cuda.current_device()) if clocks else None
    dist.barrier()
    torch.cuda.synchronize()
    ms, _ = time_steps(native, s, steps, warmup, flush, torch)
    torch.cuda.synchronize()
    dist.barrier()
    clk = sampler.stop() if sampler else None
    guard = s.sync()
    total_ms = dist.max(sum(ms), device="cuda")
    out = {"value": round(whole_job_value(world, case.ncells, steps, total_ms), 2), "steps": steps,
           "ms_per_step": round(total_ms / steps, 5), "launch": list(launch), "positivity_guard_cells": int(guard)}
    native.cteno_set_timing(s.ctx, True)
    _, kms = time_steps(native, s, max(5, min(steps, 50)), 2, flush, torch, kernel_times=True)
    native.cteno_set_timing(s.ctx, False)
    recon_ms, flux_ms = float(kms[:, 0].mean()) / 3.0, float(kms[:, 1].mean()) / 3.0
    out["roofline"] = roofline_of(case, scheme, degree, precision, launch[0], stats, recon_ms, peaks, peak_kind, alu)
    out["flux"] = {"launch_ms": round(flux_ms, 5), "algorithmic_bytes_per_launch": stats[1],
                   "achieved_gbs": round(stats[1] / (flux_ms * 1e-3) / 1e9, 1)}
    # per stage one reconstruction and one (or, face-based, two) flux/update launches; a
    # moving-shock boundary adds the time advance at the end of each step
    out["gpu_launches"] = (3 * (1 + (2 if launch[1] >= 8192 else 1)) + (1 if "regions" in case.extra else 0)) * steps
    if clk is not None:
        out["clocks"] = clk
    if e2e:
        nv = case.dim + 2
        hin = torch.empty(nv * case.ncells, dtype=torch.float64, pin_memory=True)
        hout = torch.empty(nv * case.ncells, dtype=torch.float64, pin_memory=True)
        pinned, outs = hin.numpy(), hout.numpy()
        native.cteno_get_state_all(s.ctx, pinned)
        n_e2e = max(5, min(steps, 50))
        torch.cuda.synchronize()
        t_total = 0.0
        parts = np.zeros(3)  # state in (host -> device), the step, state out (device -> host), ms
        for it in range(n_e2e + 2):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record()
            native.cteno_set_state_all(s.ctx, pinned)
            ev[1].record()
            s.run(1)
            ev[2].record()
            native.cteno_get_state_all(s.ctx, outs)
            ev[3].record()
            ev[3].synchronize()
            if it >= 2:
                t_total += ev[0].elapsed_time(ev[3])
                parts += [ev[j].elapsed_time(ev[j + 1]) for j in range(3)]
        t_total = dist.max(t_total, device="cuda")
        parts /= n_e2e
        # the same bytes as one plain copy-engine transfer each way, for comparison
        dev = torch.empty(pinned.size, dtype=torch.float64, device="cuda")
        copy_ms = np.zeros(2)
        for it in range(7):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            dev.copy_(hin, non_blocking=True)
            ev[1].record()
            hout.copy_(dev, non_blocking=True)
            ev[2].record()
            ev[2].synchronize()
            if it >= 2:
                copy_ms += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])]
        copy_ms /= 5
        del dev
        out["e2e"] = {"value": round(whole_job_value(world, case.ncells, n_e2e, t_total), 2), "unit": UNIT,
                      "h2d_bytes_per_step": int(pinned.nbytes), "d2h_bytes_per_step": int(outs.nbytes),
                      "steps": n_e2e,
                      "api": "cteno_set_state_all(host) + cteno_run(1) + cteno_get_state_all(host), pinned buffers",
                      # where the end-to-end step goes: each call timed with events on the same stream;
                      # the state calls' rates are host-link rates (the kernels access the page-locked
                      # buffers directly, permuting to and from the library's cell order on the way)
                      "ms_state_in": round(float(parts[0]), 4), "ms_step": round(float(parts[1]), 4),
                      "ms_state_out": round(float(parts[2]), 4),
                      "h2d_gbs": round(pinned.nbytes / (parts[0] * 1e-3) / 1e9, 1),
                      "d2h_gbs": round(outs.nbytes / (parts[2] * 1e-3) / 1e9, 1),
                      "copy_engine_h2d_gbs": round(pinned.nbytes / (copy_ms[0] * 1e-3) / 1e9, 1),
                      "copy_engine_d2h_gbs": round(outs.nbytes / (copy_ms[1] * 1e-3) / 1e9, 1)}
    s.close()
    return out


def run_ours(args, rank, world, local):
    import torch

    from paper_2312_17042_gb300 import build as B, native

    B.build()
    torch.cuda.set_device(local)
    dist = Dist(world, "nccl")
    stream = torch.cuda.current_stream().cuda_stream
    case = make_case(args.workload, args.n)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    peaks, peak_kind = measured_peaks()
    h = dict(scheme=case.scheme, degree=case.degree, precision=args.precision)
    launch = tuple(int(x) for x in args.launch.split(",")) if args.launch else None

    if args.profile:   # headline only: warm-up + steps, nothing else (a short command for ncu)
        s = make_solver(native, case, h["scheme"], h["degree"], h["precision"], stream)
        if launch:
            native.cteno_set_launch(s.ctx, *launch)
        else:
            launch = native.cteno_autotune(s.ctx)
            native.cteno_set_state_all(s.ctx, case.states)
        time_steps(native, s, args.steps, args.warmup, flush, torch)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.workload, "launch": launch, "guard": s.sync()}))
        s.close()
        dist.close()
        return

    alu = alu_peak(native)
    head = measure(native, case, h["scheme"], h["degree"], h["precision"], stream, flush, torch, dist, world,
                   args.steps, args.warmup, peaks, peak_kind, alu, launch=launch, clocks=True, e2e=True)

    # variants: the headline workload in the other precision, then every other configuration ----
    variants = {}
    if args.variants != "none":
        plan = [(case, sc, dg, pr) for sc, dg in case.variants for pr in (1, 0)
                if (sc, dg, pr) != (h["scheme"], h["degree"], h["precision"])]
        for other in WORKLOADS:
            if other != case.name and args.variants == "all":
                plan.append((other, None, None, None))
        for item in plan:
            if isinstance(item[0], str):
                oc = make_case(item[0])
                for sc, dg in oc.variants:
                    for pr in (1, 0):
                        variants[f"{oc.name}:{variant_name(sc, dg, pr)}"] = measure(
                            native, oc, sc, dg, pr, stream, flush, torch, dist, world, 0, 3, peaks, peak_kind,
                            alu, seconds=args.variant_seconds)
                for sc, dg in oc.variants:
                    m = variants[f"{oc.name}:{variant_name(sc, dg, 1)}"]
                    m["speedup_vs_fp64"] = round(m["value"] / variants[f"{oc.name}:{variant_name(sc, dg, 0)}"]["value"], 2)
                    m["config"] = oc.description
                del oc
            else:
                oc, sc, dg, pr = item
                variants[f"{oc.name}:{variant_name(sc, dg, pr)}"] = measure(
                    native, oc, sc, dg, pr, stream, flush, torch, dist, world, 0, 3, peaks, peak_kind, alu,
                    seconds=args.variant_seconds)
    # the cost comparison of the paper's Tables 4-5 (time per step normalised to CWENO of the same
    # order), per workload, degree and precision on the GPU
    timed = dict(variants)
    timed[f"{case.name}:{variant_name(h['scheme'], h['degree'], h['precision'])}"] = head
    for name in {k.split(":")[0] for k in timed}:
        for dg in range(2, 7):
            for pr in (0, 1):
                base = timed.get(f"{name}:{variant_name(2, dg, pr)}")
                if not base:
                    continue
                for sc in (2, 3, 0, 1):
                    v = timed.get(f"{name}:{variant_name(sc, dg, pr)}")
                    if v:
                        v["time_vs_cweno_same_order"] = round(v["ms_per_step"] / base["ms_per_step"], 3)
    fp64_same = variants.get(f"{case.name}:{variant_name(h['scheme'], h['degree'], 0)}")

    # CPU baseline: the oracle on the host cores -------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample_timing(case, h)

    result = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": head["steps"],
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (reconstruction, flux) + f64 (accumulation)" if h["precision"] else "f64",
        "data": "synthetic (seeded jittered simplex meshes, analytic initial data)",
        "config": {"workload": case.description, "scheme": SCHEMES[h["scheme"]], "degree": h["degree"],
                   "precision": PRECISIONS[h["precision"]], "cells": case.ncells,
                   "l2": "flushed before every timed step (256 MB write, untimed)",
                   "parallelism": f"replicas x{world}", "recon_block": head["launch"][0],
                   "flux_block": head["launch"][1], "positivity_guard_cells": head["positivity_guard_cells"]},
        "roofline": head["roofline"],
        "flux_kernel": head["flux"],
        "cpu_baseline": cpu,
        "e2e": head["e2e"],
        # per stage: one reconstruction launch and one flux/update launch, or two for the
        # face-based flux schedule (face fluxes, then the per-cell update)
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
        "fp64_same_workload": ({"value": fp64_same["value"], "speedup_mixed_vs_fp64":
                                round(head["value"] / fp64_same["value"], 2)} if fp64_same else None),
        "variants": variants,
        "alu_peak_measured": alu,
    }
    dist.close()
    if rank == 0:
        print(json.dumps(result))


def _subbox_sample(case, target):
    """About `target` cells of the first mesh whose centroids lie in a cube (square) around the
    workload's sample centre, as a sorted id array (all cells when the mesh is small)."""
    import workloads as W
    mesh = case.meshes[0]
    if mesh.ncells <= target:
        return np.arange(mesh.ncells, dtype=np.int32)
    cen = W.cell_centroids(mesh)
    d = np.abs(cen - np.asarray(case.sample_centre)).max(axis=1)   # Chebyshev distance
    return np.sort(np.argsort(d, kind="stable")[:target]).astype(np.int32)


def _oracle_for(case, mesh, degree, scheme):
    """The oracle of a workload (set-up deferred to the sampled cells), with its boundary regions."""
    from oracle import Oracle
    params = {k: v for k, v in case.extra.items() if k not in ("regions", "states")}
    o = Oracle(mesh, setup=False, degree=degree, scheme=scheme, cfl=case.cfl, **params)
    for lo, hi, kind in case.extra.get("regions", ()):
        o.boundary_region(lo, hi, kind)
    if "states" in case.extra:
        o.boundary_states(*case.extra["states"])
    return o


# cells of one oracle stage of the sample, by (dim, degree): about 1-2 s of one stage on 16 cores
SAMPLE_CELLS = {(2, 2): 131072, (2, 3): 131072, (3, 2): 300000, (3, 3): 60000, (2, 4): 60000, (2, 5): 40000,
                (2, 6): 30000}


def oracle_sample_timing(case, h, budget_s=20.0):
    """The oracle, as it stands, on the host cores, on a bounded sample of the workload: RK stages
    (reconstruction, HLLC flux and residual; the RK combination is negligible) of the cells of a
    sub-box of the workload's first mesh (the whole mesh when it is small), each cell and its face
    neighbours reconstructed once per stage. Set-up of the sample excluded."""
    from oracle import Oracle, num_threads
    mesh, U0 = case.meshes[0], case.states[0]
    ids = _subbox_sample(case, SAMPLE_CELLS[(case.dim, h["degree"])])
    t0 = time.perf_counter()
    o = _oracle_for(case, mesh, h["degree"], h["scheme"])
    o.set_state(U0)
    nbr = o.geometry()["nbr"][ids]
    o.setup_cells(np.unique(np.concatenate([ids, nbr[nbr >= 0]])))
    setup = time.perf_counter() - t0
    stages, t = 0, 0.0
    while stages < 2 or (t < budget_s and stages < 20):
        t0 = time.perf_counter()
        o.residual_subset(ids)
        t += time.perf_counter() - t0
        stages += 1
    whole = ids.size == mesh.ncells
    return {"value": round(ids.size * stages / t / 1e6, 5), "unit": UNIT, "cores": num_threads(), "kind": "oracle",
            "sample": f"{stages} RK stages (reconstruction + HLLC residual) of "
                      f"{'all' if whole else 'a sub-box of'} {ids.size} cells of the {mesh.ncells}-cell first mesh, "
                      f"{SCHEMES[h['scheme']]} degree {h['degree']}, FP64; set-up of the sample ({setup:.1f} s) excluded"}


# ------------------------------------------------------------------------------------------------
# reference arm: the oracle, timed as it stands on the host cores
# ------------------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import Oracle, num_threads
    case = make_case(args.workload, args.n)
    h = dict(scheme=case.scheme, degree=case.degree)
    mesh, U0 = case.meshes[0], case.states[0]
    ids = _subbox_sample(case, SAMPLE_CELLS[(case.dim, case.degree)])
    o = _oracle_for(case, mesh, case.degree, case.scheme)
    o.set_state(U0)
    nbr = o.geometry()["nbr"][ids]
    o.setup_cells(np.unique(np.concatenate([ids, nbr[nbr >= 0]])))
    # each step is one RK stage of the sample; the number of timed steps is capped so the run
    # stays within about a minute
    t0 = time.perf_counter()
    o.residual_subset(ids)
    per = time.perf_counter() - t0
    steps = max(1, min(args.steps, int(60.0 / max(per, 1e-3))))
    warm = min(args.warmup, 1)
    for _ in range(warm):
        o.residual_subset(ids)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.residual_subset(ids)
    t = time.perf_counter() - t0
    value = ids.size * steps / t / 1e6
    whole = ids.size == mesh.ncells
    sample = (f"{steps} RK stages (of {args.steps} requested steps, capped to ~1 min; reconstruction + HLLC "
              f"residual) of {'all' if whole else 'a sub-box of'} {ids.size} cells of the {mesh.ncells}-cell "
              f"first mesh, {SCHEMES[case.scheme]} degree {case.degree}, FP64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": round(t / steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case.description, "scheme": SCHEMES[case.scheme], "degree": case.degree},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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
