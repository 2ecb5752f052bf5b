"""The arithmetic behind bench.py's roofline fields, on synthetic timings
(no GPU): achieved rates follow from the stated work per DOF, the DOF one
launch processes and the mean launch time; the headline roofline is the whole
step's algorithmic bytes (16 per DOF in FP32) over ms_per_step against the
HBM peak; the dominant kernel is the one with the most time per step."""
import importlib.util
import os
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_math_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _mesh(n_cells, n_faces, n_boundary):
    nb = np.zeros(n_faces, dtype=np.int64)
    nb[:n_boundary] = -1
    return types.SimpleNamespace(n_cells=n_cells, n_faces=n_faces, face_neighbor=nb)


def test_per_kernel_rates_and_the_dominant_kernel(bench, monkeypatch):
    monkeypatch.setattr(bench, "recorded_traffic", lambda: {})   # no ncu record
    mesh = _mesh(1000, 2100, 100)                    # 2 x 2100 - 100 = 4100 incidences: 4.1 per cell
    grid = types.SimpleNamespace(n_v=4096)
    dof, steps = mesh.n_cells * grid.n_v, 10
    # (ms in total, launches) over the 10 steps: 16 blocks per step
    stats = {"block_reconstruction": (200.0, 160), "block_fluxes": (150.0, 160), "block_stage1": (80.0, 160),
             "stage2": (100.0, 10), "velocity_block_sweep": (540.0, 10)}
    ms_per_step = 55.0
    roofline, kernels, step = bench.rooflines(stats, mesh, grid, dof, steps, ms_per_step)
    hbm_peak, _, fp32_peak = bench.load_peaks()
    inc = 4100 / 1000
    k = kernels["block_reconstruction"]
    launch_s = 200.0 / 160 * 1e-3
    dof_launch = dof * steps / 160
    assert k["flops_per_dof"] == pytest.approx(41 + 31 * inc)
    assert k["alu_tflops"] == pytest.approx((41 + 31 * inc) * dof_launch / launch_s / 1e12)
    assert k["alu_frac"] == pytest.approx(k["alu_tflops"] / fp32_peak)
    s2 = kernels["stage2"]
    assert s2["bytes_per_dof"] == 8                  # read f~, write f^{n+1} in FP32
    assert s2["hbm_gbs"] == pytest.approx(8 * dof / (100.0 / 10 * 1e-3) / 1e9)
    assert s2["hbm_frac"] == pytest.approx(s2["hbm_gbs"] / hbm_peak)
    # headline: 16 B per DOF over ms_per_step against the HBM peak
    assert roofline["bound"] == "hbm" and roofline["unit"] == "GB/s"
    assert roofline["achieved"] == pytest.approx(16 * dof / (ms_per_step * 1e-3) / 1e9)
    assert roofline["frac"] == pytest.approx(roofline["achieved"] / hbm_peak)
    assert roofline["algorithmic_bytes_per_step"] == 16 * dof
    # the reconstruction has the most time per step: it is the dominant kernel;
    # without measured DRAM bytes it carries no algorithmic bytes and is ALU-bound
    assert step["dominant_kernel"] == "block_reconstruction" and k["bound"] == "alu"
    # whole step: 16 B per DOF against HBM, the sum of the kernels' flops against FP32
    t = 540.0 / 10 * 1e-3
    assert step["hbm"]["achieved_gbs"] == pytest.approx(16 * dof / t / 1e9)
    assert step["alu"]["flops_per_dof"] == pytest.approx(sum(v["flops_per_dof"] for v in kernels.values()))


def test_measured_dram_bytes_set_the_kernel_bound_and_step_traffic(bench, monkeypatch):
    mesh = _mesh(1000, 2100, 100)
    grid = types.SimpleNamespace(n_v=4096)
    dof, steps = mesh.n_cells * grid.n_v, 10
    stats = {"block_reconstruction": (200.0, 160), "block_fluxes": (150.0, 160), "block_stage1": (80.0, 160),
             "stage2": (100.0, 10), "velocity_block_sweep": (540.0, 10)}
    # DRAM bytes per launch far above what the ALU time covers at the peaks
    dram = {"block_reconstruction": 4e9, "block_fluxes": 1e6, "block_stage1": 2e6, "stage2": 3e7}
    monkeypatch.setattr(bench, "recorded_traffic", lambda: dram)
    roofline, kernels, _ = bench.rooflines(stats, mesh, grid, dof, steps, 55.0)
    hbm_peak, _, _ = bench.load_peaks()
    k = kernels["block_reconstruction"]
    assert k["dram_gbs"] == pytest.approx(4e9 / (200.0 / 160 * 1e-3) / 1e9)
    assert k["dram_frac"] == pytest.approx(k["dram_gbs"] / hbm_peak)
    assert k["bound"] == "hbm" and kernels["block_fluxes"]["bound"] == "alu"
    # per step: 16 launches of each block kernel, one second stage
    assert roofline["traffic"] == pytest.approx(16 * (4e9 + 1e6 + 2e6) + 3e7)


def test_launch_count_of_the_blocked_sweep(bench):
    stats = {"cell_stage": (1.0, 3), "face_stage": (1.0, 3), "velocity_block_sweep": (1.0, 3),
             "block_reconstruction": (1.0, 384), "block_fluxes": (1.0, 384), "block_stage1": (1.0, 384),
             "conserve": (1.0, 3), "stage2": (1.0, 3), "residual": (1.0, 3)}
    # per step: 1 + 1 + 1 + 3 x 128 + 2 + 3 + 1 = 393 launches
    assert bench.count_launches(stats) == 3 * 393
    fused = {"cell_stage": (1.0, 3), "face_stage": (1.0, 3), "velocity_block_sweep": (1.0, 3),
             "block_reconstruction": (1.0, 384), "block_flux_stage1": (1.0, 384),
             "conserve": (1.0, 3), "stage2": (1.0, 3), "residual": (1.0, 3)}
    # per step: 1 + 1 + 1 + 2 x 128 + 2 + 3 + 1 = 265 launches
    assert bench.count_launches(fused) == 3 * 265


def test_batch_workload_inputs(bench):
    """The cylinder batch: Ma in [2, 8], Kn in [1e-3, 1], 5k-40k cells,
    20^2-48^2 velocities of spacing <= 0.7, BGK, and the potential-flow start:
    uniform rho and T, speed at most u_inf, tangential to the wall, near zero
    at the rear stagnation point and u_inf far upstream."""
    from paper_2606_15720_gb300 import inputs as I
    cases = bench.batch_cases(n=3)
    for mesh, grid, gas, W0, mach, kn in cases:
        assert 2.0 <= mach <= 8.0 and 1e-3 <= kn <= 1.0
        assert 4500 <= mesh.n_cells <= 44000
        nvx = int(round(np.sqrt(grid.n_v)))
        assert nvx * nvx == grid.n_v and 20 <= nvx <= 48
        assert grid.u[1, 0] - grid.u[0, 0] <= 0.7 + 1e-12 or nvx == 48
        assert gas.model == "bgk"
        u_inf = mesh.bc[1].u[0]
        prim = I.cylinder_potential_primitives(mesh, u_inf)
        np.testing.assert_allclose(W0, I.prim_to_conservative(prim, 2, 0))
        assert np.all(prim[:, 0] == 1.0) and np.all(prim[:, 3] == 1.0)
        speed = np.linalg.norm(prim[:, 1:3], axis=1)
        assert np.max(speed) <= u_inf * (1 + 1e-12)
        x = mesh.cell_centroid
        r = np.linalg.norm(x, axis=1)
        near = r < 0.56
        un = np.abs(np.sum(prim[near, 1:3] * x[near], axis=1) / r[near])
        assert np.max(un / u_inf) < 0.25                   # O(r - R) next to the wall
        rear = np.argmin(np.linalg.norm(x - np.array([0.5, 0.0]), axis=1))
        assert speed[rear] < 0.2 * u_inf
        far = np.argmin(x[:, 0])
        assert speed[far] == pytest.approx(u_inf, rel=0.02)
    # lateral edges are outflow, the inflow edge far field
    mesh = cases[0][0]
    nb = mesh.face_neighbor
    bnd = nb < 0
    bc = -(nb[bnd] + 1)
    yc = mesh.face_centroid[bnd, 1]
    xc = mesh.face_centroid[bnd, 0]
    assert np.all(bc[np.abs(np.abs(yc) - 5.0) < 1e-9] == 2)
    assert np.all(bc[np.abs(xc + 4.0) < 1e-9] == 1)
