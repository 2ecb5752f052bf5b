"""Benchmark of the UGKS velocity-block sweep on the 3-D sphere workload.

Workload: hypersonic flow (Ma 5, Kn 0.05, Shakhov, Pr 2/3, monatomic) around a
unit sphere on a seeded Delaunay tetrahedral mesh of ~1e5 cells graded toward
the body, with a 32^3 uniform velocity grid on [-12, 12]^3 (3.3e9 phase-space
points), FP32 distribution storage with FP64 moments, W update and interface
coefficients; diffuse isothermal wall at the stagnation temperature.  Inputs
are synthetic (no dataset).

metric: phase-space DOF updates per second = n_cells * n_v * n_reduced / step time.

Arms:
  default            the CUDA library through its C ABI; device-timed steps
                     (CUDA events on the library's stream), plus an end-to-end
                     number through the one-shot host-buffer call, a roofline
                     for the sweep kernel and the oracle's CPU baseline.
  --impl reference   the FP64 CPU oracle on a bounded sample of the workload.
Under torchrun each rank runs an independent replica (the path does not shard
across GPUs); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_15720_gb300 import inputs as I  # noqa: E402

METRIC = "phase-space DOF updates/s per UGKS step"
UNIT = "DOF/s"
WORKLOAD = "sphere_tet100k_v32cube_shakhov_ma5_kn0.05_fp32"
MESH_CELLS = 100_000
MESH_SEED = 2
NV_AXIS = 32


def build_workload(cells=MESH_CELLS, nv_axis=NV_AXIS, nv_cross=0):
    mesh = I.sphere_tet_mesh(cells, seed=MESH_SEED)
    n = [nv_axis, nv_cross, nv_cross] if nv_cross > 0 else nv_axis
    grid = I.midpoint_grid(n, -12.0, 12.0, 3)
    gas = I.Gas(model="shakhov", K=0, Pr=2.0 / 3.0, omega=0.81, mu_ref=I.mu_ref_from_kn(0.05, 0.81), cfl=0.8)
    prim = I.uniform_primitives(mesh, 1.0, mesh.bc[1].u, 1.0)   # freestream start
    W0 = I.prim_to_conservative(prim, 3, 0)
    return mesh, grid, gas, W0


def workload_config(mesh, grid, gas, world, workload=WORKLOAD, sweep="auto", storage="f32", block_velocities=0):
    """The benchmark's config entry, the same for the CUDA arm and the
    reference (oracle) arm: the workload and its sizes."""
    n_reduced = 2 if gas.K + 3 - mesh.dim > 0 else 1
    dof = mesh.n_cells * grid.n_v * n_reduced
    return {"workload": workload, "n_cells": mesh.n_cells, "n_faces": mesh.n_faces, "n_v": grid.n_v,
            "n_reduced": n_reduced, "dof_per_step": dof, "parallelism": f"replicas x{world}",
            "sweep": sweep, "storage": storage,
            "block_velocities": block_velocities or (256 if mesh.dim == 3 and gas.K == 0 else 128),
            "l2": "inputs larger than L2 (two %.1f GB distribution buffers)" % (dof * 4 / 1e9)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_timing(local_ms, steps, dof_per_replica, world, dist=None, device="cuda"):
    """Whole-job timing of N independent replicas: the slowest rank's time for
    the timed steps (max over ranks), and the DOF updates of all ranks per
    second of it.  Returns (ms per step, DOF/s)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item()) / steps
    return ms_per_step, dof_per_replica * world / (ms_per_step * 1e-3)


N_SM = 152            # GB300 multiprocessors
FP32_LANES = 128      # FP32 lanes per multiprocessor


def load_peaks():
    """HBM GB/s (measured copy) and the FP32 CUDA-core peak in TFLOP/s derived
    from unit counts and the maximum SM clock: 152 SMs x 128 lanes x 2 (FMA)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        mhz = float(d.get("sm_max_mhz", 2070.0))
        return float(d["hbm_gbs"]), "measured", N_SM * FP32_LANES * 2 * mhz * 1e6 / 1e12
    return 6800.0, "fallback", N_SM * FP32_LANES * 2 * 2070e6 / 1e12


# Algorithmic work of the blocked sweep per velocity (FP32 operations, FMA = 2,
# counted term by term from the formulas each kernel evaluates: gradient 9,
# limiter increment 7 and upwind face value 15 per face, 41 per velocity (two
# limiter evaluations, the limiter constants, clipping, scaling, u.g) in the
# reconstruction; 69 per face-velocity in the flux; 27 + 2 per face in the
# first stage; 34 in the second).  inc = faces per cell (4 on tetrahedra).
def flops_recon(inc):       # per cell-velocity: LSQ gradient, limiter, upwind face values
    return 41 + 31 * inc


FLOPS_FLUX = 69             # per face-velocity: upwind pick, g0 P(c), flux, moments


def flops_stage1(inc):      # per cell-velocity
    return 27 + 2 * inc


FLOPS_STAGE2 = 34           # per cell-velocity
BYTES_STAGE = 8             # per DOF and stage update: read + write of an FP32 f value
BYTES_STAGE_SCALED = 2 * (2 + 4 / 32)   # FP16 / BF16 value + its row's FP32 scale, read + write


def sweep_source_hash():
    h = hashlib.sha256()
    for fn in ("ugks_blocked.cuh", "ugks_bulk.cuh", "ugks_internal.cuh", "ugks_kernels.cuh", "ugks_device.cuh"):
        with open(os.path.join(ROOT, "paper_2606_15720_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of each blocked-sweep kernel from the committed
    ncu summary, if it was taken on the current kernel source (else {})."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        d = json.load(fh)
    if d.get("source_hash") != sweep_source_hash():
        return {}
    return d.get("dram_bytes_per_launch", {})


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(mesh, grid, gas, W0, dt, target_cells=3000, steps=6):
    """The FP64 oracle as it stands, on a bounded sample of the workload: the
    face-connected patch of ~target_cells cells around a body-adjacent cell,
    all 32^3 velocities, `steps` steps at the GPU run's time step dt."""
    import oracle as O
    seed = int(mesh.face_owner[np.flatnonzero(mesh.face_neighbor == -1)[0]])
    rings, cells, pm = 1, None, None
    while True:
        cells, pm = I.submesh(mesh, [seed], rings)
        if pm.n_cells >= target_cells or rings > 40:
            break
        rings += 1
    W = W0[cells]
    f = O.initial_f(pm, grid, W, gas.K)
    O.run(pm, grid, gas, W, f, 1, dt=dt)             # warm-up (page-in, thread pool)
    t0 = time.perf_counter()
    O.run(pm, grid, gas, W, f, steps, dt=dt)
    el = time.perf_counter() - t0
    dof = pm.n_cells * grid.n_v * O.n_reduced(3, gas.K)
    out = {"value": dof * steps / el, "unit": UNIT, "cores": O.num_threads(), "cpu_model": cpu_model(),
           "nproc": os.cpu_count(), "kind": "oracle", "dt": dt,
           "sample": f"{steps} steps of a {pm.n_cells}-cell patch of the workload mesh x {grid.n_v} velocities "
                     f"at the GPU run's dt ({dof * steps:.3g} DOF updates, {el:.1f} s)"}
    # one thread, on a patch of about a tenth of the cells
    rings, cells1, pm1 = 1, None, None
    while True:
        cells1, pm1 = I.submesh(mesh, [seed], rings)
        if pm1.n_cells >= target_cells // 10 or rings > 40:
            break
        rings += 1
    W1 = W0[cells1]
    f1 = O.initial_f(pm1, grid, W1, gas.K)
    prev = O.set_threads(1)
    try:
        t0 = time.perf_counter()
        O.run(pm1, grid, gas, W1, f1, 2, dt=dt)
        el1 = time.perf_counter() - t0
    finally:
        O.set_threads(prev)
    dof1 = pm1.n_cells * grid.n_v * O.n_reduced(3, gas.K)
    out["single_thread"] = {"value": dof1 * 2 / el1, "unit": UNIT, "cores": 1,
                            "sample": f"2 steps of a {pm1.n_cells}-cell patch x {grid.n_v} velocities ({el1:.1f} s)"}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    mesh, grid, gas, W0 = build_workload()
    import oracle as O
    seed = int(mesh.face_owner[np.flatnonzero(mesh.face_neighbor == -1)[0]])
    rings = 1
    while True:
        cells, pm = I.submesh(mesh, [seed], rings)
        if pm.n_cells >= 1500 or rings > 40:
            break
        rings += 1
    W = W0[cells]
    f = O.initial_f(pm, grid, W, gas.K)
    dt = O.time_step(mesh, grid, gas.cfl)          # the time step of the full workload
    dof = pm.n_cells * grid.n_v * O.n_reduced(3, gas.K)
    for _ in range(args.warmup):
        W, f, _, _ = O.run(pm, grid, gas, W, f, 1, dt=dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W, f, _, _ = O.run(pm, grid, gas, W, f, 1, dt=dt)
    el = time.perf_counter() - t0
    value = dof * args.steps / el
    sample = (f"each step: one oracle step of a {pm.n_cells}-cell face-connected patch of the {mesh.n_cells}-cell "
              f"workload mesh x {grid.n_v} velocities; value = the patch's DOF updates per second")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp64", "data": "synthetic",
            "config": workload_config(mesh, grid, gas, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "cpu_model": cpu_model(),
                             "nproc": os.cpu_count(), "kind": "oracle", "dt": dt, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def rooflines(stats, mesh, grid, dof, steps, ms_per_step, bytes_stage=BYTES_STAGE):
    """Rooflines of the blocked sweep from the library's event timings (CUDA
    events on the stream the kernels run on).

    roofline (the headline): the whole step against HBM on its algorithmic
    bytes: 4 s bytes per phase-space DOF (s = bytes per stored
    value: the first stage reads f^n and writes f~, the second reads f~ and
    writes f^{n+1}), achieved = 4 s x DOF / (ms_per_step), so the fraction
    reproduces from ms_per_step.  traffic = the step's DRAM bytes from the
    committed ncu capture (null when the kernels changed since).
    kernels: per kernel the ALU view (algorithmic FP32 operations), the
    algorithmic-bytes view where the kernel has algorithmic bytes, and the
    measured DRAM rate (ncu bytes per launch / event-timed launch); the bound
    is the larger of the two times at the peaks, using the measured bytes
    where they exist."""
    hbm_peak, peak_kind, fp32_peak = load_peaks()
    n_inc = 2 * mesh.n_faces - int(np.sum(mesh.face_neighbor < 0))
    inc = n_inc / mesh.n_cells
    traffic = recorded_traffic()
    fpc = mesh.n_faces / mesh.n_cells
    per_dof = {"block_reconstruction": (flops_recon(inc), 0), "block_fluxes": (FLOPS_FLUX * fpc, 0),
               "block_stage1": (flops_stage1(inc), bytes_stage),
               # fused flux + first stage: the algorithmic flops of both (each face counted once)
               "block_flux_stage1": (FLOPS_FLUX * fpc + flops_stage1(inc), bytes_stage),
               "stage2": (FLOPS_STAGE2, bytes_stage)}
    kernels = {}
    step_traffic, traffic_complete = 0.0, bool(traffic)
    for name, (fl, by) in per_dof.items():
        ms, n = stats.get(name, (0.0, 0))
        if not n:
            continue
        launch_s = ms / n * 1e-3
        dof_launch = dof * steps / n              # phase-space points one launch processes
        tflops = fl * dof_launch / launch_s / 1e12
        gbs = by * dof_launch / launch_s / 1e9
        dram = traffic.get(name)
        if dram is None:
            traffic_complete = False
        else:
            step_traffic += dram * n / steps
        dram_gbs = dram / launch_s / 1e9 if dram is not None else None
        t_alu = fl * dof_launch / (fp32_peak * 1e12)
        t_mem = (dram if dram is not None else by * dof_launch) / (hbm_peak * 1e9)
        kernels[name] = {"launch_ms": ms / n, "ms_per_step": ms / steps, "launches_per_step": n / steps,
                         "bound": "hbm" if t_mem > t_alu else "alu",
                         "flops_per_dof": fl, "bytes_per_dof": by,
                         "alu_tflops": tflops, "alu_frac": tflops / fp32_peak,
                         "hbm_gbs": gbs if by else None, "hbm_frac": gbs / hbm_peak if by else None,
                         "dram_bytes_per_launch": dram, "dram_gbs": dram_gbs,
                         "dram_frac": dram_gbs / hbm_peak if dram_gbs is not None else None}
    b_step = 2 * bytes_stage
    achieved = b_step * dof / (ms_per_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "whole step (every kernel of one UGKS step)",
                "achieved": achieved, "peak": hbm_peak, "peak_kind": peak_kind + " (copy bandwidth)",
                "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": step_traffic if traffic_complete else None,
                "traffic_unit": "DRAM bytes per step (ncu, sum over the sweep kernels)",
                "algorithmic_bytes_per_step": b_step * dof, "bytes_per_dof": b_step,
                "launch_ms": ms_per_step}
    sweep_ms, sweep_n = stats.get("velocity_block_sweep", (0.0, 0))
    step_views = None
    if sweep_n:
        t = sweep_ms / sweep_n * 1e-3
        fl = sum(v["flops_per_dof"] for v in kernels.values())
        step_views = {"sweep_ms": sweep_ms / sweep_n,
                      "hbm": {"bytes_per_dof": b_step, "achieved_gbs": b_step * dof / t / 1e9,
                              "frac": b_step * dof / t / 1e9 / hbm_peak, "peak": hbm_peak, "peak_kind": peak_kind},
                      "alu": {"flops_per_dof": fl, "achieved_tflops": fl * dof / t / 1e12,
                              "frac": fl * dof / t / 1e12 / fp32_peak, "peak": fp32_peak,
                              "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}}
        if kernels:
            top = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
            step_views["dominant_kernel"] = top
    return roofline, kernels, step_views


def count_launches(stats):
    """Kernel launches of the library in the timed region, from its per-region
    event counts (the regions of the blocked sweep that span several kernels
    count each)."""
    if stats.get("block_reconstruction", (0, 0))[1]:
        # velocity_block_sweep: the per-cell equilibrium records; conserve: wall
        # density + W update; stage2: the second stage's two launches (CTAs
        # without and with wall cells) + heat-flux chunk sum
        per = {"cell_stage": 1, "face_stage": 1, "velocity_block_sweep": 1, "block_reconstruction": 1,
               "block_fluxes": 1, "block_stage1": 1, "block_flux_stage1": 1, "conserve": 2, "stage2": 3,
               "residual": 1}
    else:
        per = {"cell_stage": 1, "face_stage": 1, "velocity_block_sweep": 1, "residual": 1}
    return int(sum(per.get(k, 0) * n for k, (_, n) in stats.items()))


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2606_15720_gb300 import ugks as U

    mesh, grid, gas, W0 = build_workload(args.cells, args.nv_axis, args.nv_cross)
    stream = torch.cuda.Stream()
    n_reduced = 1
    dof = mesh.n_cells * grid.n_v * n_reduced

    def barrier():
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        solver = U.Solver(mesh, grid, gas, W0, storage=args.storage, stream=int(stream.cuda_stream),
                          sweep=args.sweep, block_velocities=args.block_velocities)
        assert solver.n_reduced == n_reduced
        dt_run = solver.dt
        solver.step(args.warmup)
        solver.residual()
        solver.stats_enable(True)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        start.record(stream)
        solver.step(args.steps)
        stop.record(stream)
        stop.synchronize()
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        ms = start.elapsed_time(stop)
        stats = solver.stats()
        res = solver.residual()
        W_end = solver.moments()
        # surface quantities of the last step (pressure, shear, heat flux and
        # C_p, C_t, C_h against the far-field state)
        far = mesh.bc[1]
        t0 = time.perf_counter()
        faces, svals, scoef = solver.surface([far.rho, far.u[0], far.u[1], far.u[2], far.T])
        surface = {"n_wall_faces": int(len(faces)), "ms": 1e3 * (time.perf_counter() - t0),
                   "max_Cp": float(np.max(scoef[:, 0])), "max_Ch": float(np.max(scoef[:, 2])),
                   "max_Ct": float(np.max(scoef[:, 1]))}
        solver.close()
    ms_per_step, value = replica_timing(ms, args.steps, dof, world, dist, "cuda")

    roofline, kernels, step_views = rooflines(stats, mesh, grid, dof, args.steps, ms_per_step,
                                              BYTES_STAGE if args.storage == "f32" else BYTES_STAGE_SCALED)

    # end to end through the one-shot C call with host buffers: mesh, grid and
    # W_init copied in, n steps, W and the residual copied out
    if args.no_e2e:
        e2e = None
    barrier()
    t0 = time.perf_counter()
    W_e2e, res_e2e = U.solve(mesh, grid, gas, W0, args.steps if not args.no_e2e else 0, storage=args.storage,
                             sweep=args.sweep, block_velocities=args.block_velocities)
    e2e_s = time.perf_counter() - t0
    barrier()
    in_bytes = sum(a.nbytes for a in (mesh.cell_volume, mesh.cell_centroid, mesh.face_owner, mesh.face_neighbor,
                                      mesh.face_area, mesh.face_normal, mesh.face_centroid, mesh.face_shift,
                                      grid.u, grid.weight, W0))
    out_bytes = W_e2e.nbytes + res_e2e.nbytes
    te = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = None if args.no_e2e else {"value": dof * world * args.steps / float(te.item()), "unit": UNIT,
           "h2d_bytes_per_step": int(math.ceil(in_bytes / args.steps)),
           "d2h_bytes_per_step": int(math.ceil(out_bytes / args.steps)),
           "includes": "ugks_solve: create from host arrays (renumbering, geometry, f init), all steps, W and residual read back"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = None
    full = (args.cells, args.nv_axis, args.nv_cross) == (MESH_CELLS, NV_AXIS, 0)
    if world == 1 and not args.no_cpu_baseline and full:
        cpu = cpu_baseline(mesh, grid, gas, W0, dt_run)
    workload = WORKLOAD if full else \
        (f"sphere_tet{args.cells // 1000}k_v{args.nv_axis}x{args.nv_cross}x{args.nv_cross}_shakhov_fp32"
         if args.nv_cross > 0 else f"sphere_tet{args.cells // 1000}k_v{args.nv_axis}cube_shakhov_fp32") + \
        " (reduced size for profiling)"
    if args.storage != "f32":
        workload = workload.replace("fp32", args.storage + "_scaled_storage")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32" if args.storage == "f32" else f"fp32 arithmetic, {args.storage} storage",
            "data": "synthetic",
            "config": workload_config(mesh, grid, gas, world, workload, args.sweep, args.storage,
                                      args.block_velocities),
            "state_after": {"residual": [float(x) for x in res], "finite": bool(np.all(np.isfinite(W_end)))},
            "roofline": roofline, "kernels": kernels, "step_roofline": step_views,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": count_launches(stats),
            "surface": surface,
            "kernel_ms": {k: v[0] / max(v[1], 1) for k, v in stats.items()},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_mixed_report(args):
    """Per-field error of FP32 arithmetic with FP32, FP16 and BF16 storage
    against the FP64 oracle after 100 and 1000 steps, on a reduced instance
    of the sphere workload (the same generator at 2500 cells, 24^3 velocities
    on [-12, 12]^3; the oracle cannot step the full one 1000 times).  Relative L-inf per field:
    density, momentum (as a vector), energy, temperature."""
    import oracle as O
    from paper_2606_15720_gb300 import ugks as U
    mesh = I.sphere_tet_mesh(2500, seed=MESH_SEED)
    grid = I.midpoint_grid(24, -12.0, 12.0, 3)
    gas = I.Gas(model="shakhov", K=0, Pr=2.0 / 3.0, omega=0.81, mu_ref=I.mu_ref_from_kn(0.05, 0.81), cfl=0.8)
    W0 = I.prim_to_conservative(I.uniform_primitives(mesh, 1.0, mesh.bc[1].u, 1.0), 3, 0)
    f0 = O.initial_f(mesh, grid, W0, gas.K)
    with U.Solver(mesh, grid, gas, W0, storage="f64") as s:
        dt = s.dt
    t0 = time.perf_counter()
    W100, f100, _, _ = O.run(mesh, grid, gas, W0, f0, 100, dt=dt)
    W1000, _, _, _ = O.run(mesh, grid, gas, W100, f100, 900, dt=dt)
    oracle_s = time.perf_counter() - t0
    ref = {100: W100, 1000: W1000}

    def fields(W):
        rho = W[:, 0]
        mom = W[:, 1:4]
        E = W[:, 4]
        T = 4.0 * (E - 0.5 * np.sum(mom ** 2, axis=1) / rho) / (3.0 * rho)   # K = 0, R = 1/2
        return rho, mom, E, T

    out = {}
    for st in ("f32", "f16", "bf16"):
        out[st] = {}
        with U.Solver(mesh, grid, gas, W0, storage=st) as s:
            done = 0
            for n in (100, 1000):
                s.step(n - done)
                done = n
                g, o = fields(s.moments()), fields(ref[n])
                mom_scale = np.max(np.linalg.norm(o[1], axis=1))
                out[st][str(n)] = {
                    "rho": float(np.max(np.abs(g[0] - o[0])) / np.max(np.abs(o[0]))),
                    "momentum": float(np.max(np.linalg.norm(g[1] - o[1], axis=1)) / mom_scale),
                    "energy": float(np.max(np.abs(g[2] - o[2])) / np.max(np.abs(o[2]))),
                    "temperature": float(np.max(np.abs(g[3] - o[3])) / np.max(np.abs(o[3])))}
    print(json.dumps({"report": "mixed_precision_error", "metric": "relative L-inf per field vs the FP64 oracle",
                      "config": {"workload": "sphere_tet2.5k_v24cube_shakhov_ma5_kn0.05", "n_cells": mesh.n_cells,
                                 "n_v": grid.n_v, "dt": dt, "oracle_seconds": oracle_s},
                      "errors": out}), flush=True)
    return 0


def batch_cases(n=64, seed=4, cells_range=(5e3, 4e4), nv_range=(20, 48), mach_range=(2.0, 8.0)):
    """The 64 cylinder cases of the batch workload: Ma ~ U[2, 8], Kn ~
    log-uniform [1e-3, 1], triangle meshes of 5k-40k cells (log-uniform),
    velocity grids sized to Ma (20^2 .. 48^2 points on [-v, v]^2, v covering
    the free stream and the stagnation temperature, spacing at most 0.7 =
    about the thermal width sqrt(T_inf/2) of the free stream: grids of
    spacing ~1 under-resolve the free-stream Maxwellian and those cases went
    non-physical within 40-80 steps).  Choices that keep every case physical
    over thousands of steps (each tried on the GPU in FP32 and FP64, the
    failures identical in both):
    * BGK collisions (the workload names no model): with the Shakhov
      correction, rarefied cases above Ma ~5 (Kn >= 0.05) drive f negative
      in the near-vacuum wake within 250-1000 steps;
    * the potential-flow start of inputs.cylinder_potential_primitives
      instead of a uniform free stream, which empties the cells behind the
      cylinder to ~1e-6 of the free-stream density within 100-200 steps;
    * Venkatakrishnan's limiter with K_v = 1 (eps^2 = h^3 m^2): with K_v = 5
      the coarse cells barely limit f at the bow shock;
    * outflow (zero-gradient) lateral edges (inputs.cylinder_tri_mesh)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        mach = float(rng.uniform(*mach_range))
        kn = float(10 ** rng.uniform(-3.0, 0.0))
        cells = int(round(10 ** rng.uniform(math.log10(cells_range[0]), math.log10(cells_range[1]))))
        mesh = I.cylinder_tri_mesh(cells, seed=seed * 1000 + i, mach=mach)
        u_inf = mesh.bc[1].u[0]
        T_stag = 1.0 + mach * mach / 3.0
        vmax = max(u_inf + 4.0, 3.5 * math.sqrt(T_stag))
        nvx = int(min(nv_range[1], max(nv_range[0], math.ceil(2.0 * vmax / 0.7))))
        grid = I.midpoint_grid(nvx, -vmax, vmax, 2)
        gas = I.Gas(model="bgk", K=0, Pr=1.0, omega=0.81, mu_ref=I.mu_ref_from_kn(kn, 0.81), cfl=0.8, venkat_K=1.0)
        W0 = I.prim_to_conservative(I.cylinder_potential_primitives(mesh, u_inf), 2, 0)
        out.append((mesh, grid, gas, W0, mach, kn))
    return out


def run_batch_report(args):
    """Batch workload: 64 uneven 2-D cylinder cases advanced by one CUDA-graph
    launch per two steps after the shape autotuner, against the same cases
    stepped with ordinary launches (in turn without waiting, each case on its
    own stream, and one case at a time); also 64 small cases (Ma 1.5-3,
    300-1500 cells, 20^2-24^2 velocities), where launch overhead and idle SMs
    matter."""
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU path)")
    big = time_batch(args, batch_cases(), "cylinder_batch64_ma2-8_kn1e-3-1_tri5k-40k_v20-48sq_bgk_fp32")
    small = time_batch(args, batch_cases(seed=5, cells_range=(300, 1500), nv_range=(20, 24), mach_range=(1.5, 3.0)),
                       "cylinder_batch64_small_ma1.5-3_tri300-1500_v20-24sq_bgk_fp32")
    print(json.dumps(dict(big, small_cases=small)), flush=True)
    return 0


def time_batch(args, cases, workload):
    import torch
    from paper_2606_15720_gb300 import ugks as U
    dof = sum(c[0].n_cells * c[1].n_v * 2 for c in cases)   # 2-D, K = 0: h and b
    stream = torch.cuda.Stream()
    steps = max(2, args.steps - args.steps % 2)
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        b = U.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases],
                    storage="f32", stream=int(stream.cuda_stream))
        create_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        b.autotune()
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
        picks = [b.tuning(i)[0] for i in range(len(cases))]
        shapes = [b.shape(i) for i in range(len(cases))]
        b.step(max(2, args.warmup - args.warmup % 2))   # captures the graph
        torch.cuda.synchronize()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        b.step(steps)
        stop.record(stream)
        torch.cuda.synchronize()
        graph_ms = start.elapsed_time(stop) / steps
        # the same cases, one ordinary ugks_step after another
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for s in b.cases:
                s.step(1)
        for s in b.cases:
            s.residual()          # synchronises each case's stream
        seq_ms = 1e3 * (time.perf_counter() - t0) / steps
        # one case at a time: each case's step has finished before the next
        # case's is enqueued (no overlap between cases)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for s in b.cases:
                s.step(1)
                s.residual()
        one_ms = 1e3 * (time.perf_counter() - t0) / steps
        finite = all(bool(np.all(np.isfinite(s.moments()))) for s in b.cases)
        # time to steady: graph launches (two steps each), density residuals
        # (reading R13) read every `every` steps; per case the first step count
        # (and batch wall time) at which it fell below each threshold
        steady = None
        if args.steady_steps > 0:
            thresholds = (1e-4, 1e-5, 1e-6)
            every = 100
            reached = [[None] * len(thresholds) for _ in cases]
            failed = [None] * len(cases)      # step at which a case reported a non-physical state
            done_steps, t_all = 0, 0.0
            while done_steps < args.steady_steps:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                b.step(every)
                torch.cuda.synchronize()
                t_all += time.perf_counter() - t0
                done_steps += every
                for i, cs in enumerate(b.cases):
                    if failed[i] is not None:
                        continue
                    try:
                        r = float(cs.residual()[0])
                    except U.UGKSError:
                        failed[i] = done_steps
                        continue
                    for t, thr in enumerate(thresholds):
                        if reached[i][t] is None and r < thr:
                            reached[i][t] = (done_steps, t_all)
                if all(x[-1] is not None or failed[i] is not None for i, x in enumerate(reached)):
                    break
            steady = {"steps_run": done_steps, "seconds": t_all, "ms_per_step": 1e3 * t_all / done_steps,
                      "non_physical": [{"case": i, "mach": cases[i][4], "kn": cases[i][5], "cells": int(cases[i][0].n_cells),
                                        "by_step": failed[i]} for i in range(len(cases)) if failed[i] is not None],
                      "residual": "density residual R_rho, reading R13",
                      "reached": {f"{thr:g}": {"cases": sum(1 for x in reached if x[t] is not None),
                                               "steps_median": (float(np.median([x[t][0] for x in reached
                                                                                 if x[t] is not None]))
                                                                if any(x[t] is not None for x in reached) else None),
                                               "all_cases_seconds": (max(x[t][1] for x in reached)
                                                                     if all(x[t] is not None for x in reached)
                                                                     else None)}
                                  for t, thr in enumerate(thresholds)},
                      "per_case_steps": [[(x[t][0] if x[t] is not None else None) for t in range(len(thresholds))]
                                         for x in reached]}
        b.close()
    return {
        "report": "batch", "metric": "phase-space DOF updates/s per batch step", "unit": "DOF/s",
        "config": {"workload": workload,
                   "n_cases": len(cases), "dof_per_step": dof,
                   "cells": [int(c[0].n_cells) for c in cases], "n_v": [int(c[1].n_v) for c in cases]},
        "graph": {"value": dof / (graph_ms * 1e-3), "ms_per_step": graph_ms,
                  "note": "one CUDA-graph launch per two steps of all cases, cases on forked streams"},
        "sequential": {"value": dof / (seq_ms * 1e-3), "ms_per_step": seq_ms,
                       "note": "ugks_step per case in turn without waiting: every case has its own stream, so "
                               "the GPU overlaps the cases; host wall clock"},
        "one_case_at_a_time": {"value": dof / (one_ms * 1e-3), "ms_per_step": one_ms,
                               "note": "ugks_step per case in turn, each waited for before the next case; "
                                       "host wall clock"},
        "autotune": {"seconds": tune_s, "block_velocities": {str(v): picks.count(v) for v in sorted(set(picks))},
                     "fused": sum(1 for sh in shapes if sh["fused"]),
                     "stage2_chunks": {str(c): sum(1 for sh in shapes if sh["stage2_chunks"] == c)
                                       for c in sorted(set(sh["stage2_chunks"] for sh in shapes))},
                     "distinct_shapes": len(set((sh["block_velocities"], sh["fused"], sh["stage2_chunks"])
                                                for sh in shapes)),
                     "per_case": shapes},
        "time_to_steady": steady,
        "setup_seconds": {"create": create_s}, "finite": finite, "steps": steps}


WARM_TRAIN = [(ma, kn) for ma in (1.5, 2.0, 2.5, 3.0) for kn in (0.05, 0.15, 0.5)]
def warm_held_out(n=16, seed=5):
    """Held-out (Ma, Kn) of the warm-start report: Ma ~ U[1.6, 2.9], Kn ~
    log-uniform [0.06, 0.45], inside the training family's range."""
    rng = np.random.default_rng(seed)
    return [(round(float(rng.uniform(1.6, 2.9)), 3), round(float(10 ** rng.uniform(math.log10(0.06), math.log10(0.45))), 4))
            for _ in range(n)]


WARM_TRAIN_BATCH = [(2.0, 1e-3), (2.0, 1e-2), (2.0, 0.1), (2.0, 1.0), (3.5, 1e-3), (3.5, 1e-2), (3.5, 0.1),
                    (3.5, 1.0), (5.0, 0.03), (5.0, 0.1), (5.0, 1.0), (6.5, 0.05), (6.5, 0.15), (6.5, 1.0),
                    (8.0, 0.05), (8.0, 0.15), (8.0, 1.0)]


def warm_held_out_batch(n=8, seed=6):
    """Held-out (Ma, Kn) of the wide warm-start family: Ma ~ U[2.3, 7.7],
    Kn log-uniform in [1.5e-3, 0.7], redrawn where Ma > 4.5 and Kn < 0.05
    (the continuum corner whose strong shocks do not stay physical on
    2000-triangle meshes: Ma 5-8 at Kn 1e-3-1e-2 went non-physical within
    1500-3500 steps there)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        ma = float(rng.uniform(2.3, 7.7))
        kn = float(10 ** rng.uniform(math.log10(1.5e-3), math.log10(0.7)))
        if ma > 4.5 and kn < 0.05:
            continue
        out.append((round(ma, 3), round(kn, 4)))
    return out


def run_warm_report(args):
    """Learned warm start: 12 converged cylinder cases (Ma 1.5-3, Kn 0.05-0.5,
    about 2000 triangles, 28^2 velocities, Shakhov) train the 6x256 network;
    16 held-out cases (new meshes, Ma and Kn between the training values) are
    solved to residual 1e-6 from the freestream and from the warm start, and
    both results are compared with the freestream solve continued to 1e-8."""
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU path)")
    from paper_2606_15720_gb300 import warmstart as WS
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    if args.family == "batch":
        res = WS.experiment(WARM_TRAIN_BATCH, warm_held_out_batch(), cells=2000, nvx=None, ref_tol=1e-8,
                            max_steps=60_000, family="batch", log=log)
        res["workload"] = "cylinder_warmstart_ma2-8_kn1e-3-1_tri2k_v20-48sq_bgk_potential_start_fp32"
    else:
        res = WS.experiment(WARM_TRAIN, warm_held_out(), cells=2000, nvx=28, ref_tol=1e-8, log=log)
        res["workload"] = "cylinder_warmstart_ma1.5-3_kn0.05-0.5_tri2k_v28sq_shakhov_fp32"
    ratios = [c["time_ratio"] for c in res["cases"] if "time_ratio" in c]
    res["metric"] = "time_to_residual_1e-6_speedup"
    res["value"] = float(np.exp(np.mean(np.log(ratios)))) if ratios else None
    res["unit"] = "x (geometric mean over held-out cases, freestream seconds / warm-start seconds)"
    print(json.dumps(res), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cells", type=int, default=MESH_CELLS, help="mesh size (profiling runs only)")
    ap.add_argument("--nv-axis", type=int, default=NV_AXIS, help="velocities per axis (profiling runs only)")
    ap.add_argument("--nv-cross", type=int, default=0,
                    help="velocities along the two cross-flow axes, 0 = as --nv-axis (profiling runs only)")
    ap.add_argument("--sweep", default="auto", choices=["auto", "blocked", "blocked_fused", "tiled"])
    ap.add_argument("--block-velocities", type=int, default=0, choices=[0, 32, 64, 128, 256])
    ap.add_argument("--steady-steps", type=int, default=0,
                    help="batch report: also step the batch up to this many steps, recording time to steady")
    ap.add_argument("--family", default="shakhov", choices=["shakhov", "batch"],
                    help="warmstart report: the Ma 1.5-3 Shakhov family, or cases of the batch workload's "
                         "kind (Ma 2-8, Kn 1e-3-1, BGK, potential-flow start)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="storage of f (FP16 / BF16: deviations from a per-cell reference Maxwellian)")
    ap.add_argument("--report", default=None, choices=["mixed", "batch", "warmstart"],
                    help="mixed: per-field error of FP32/FP16/BF16 storage vs the oracle at 1e2 and 1e3 steps; "
                         "batch: 64 uneven cylinder cases in one CUDA graph with the block-size autotuner; "
                         "warmstart: time to steady residual 1e-6 from the learned warm start vs the freestream")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.report == "mixed":
        return run_mixed_report(args)
    if args.report == "batch":
        return run_batch_report(args)
    if args.report == "warmstart":
        return run_warm_report(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
