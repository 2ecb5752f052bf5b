"""C ABI: the library builds, loads and exports every entry point that
include/ugks.h declares; argument validation happens on the host before any
CUDA call, so it is checked here without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_15720_gb300 import build, inputs as I, ugks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ugks_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ugks.load()


def test_library_exports_every_declared_entry_point(lib):
    names = declared_entry_points()
    assert "ugks_create" in names and "ugks_step" in names and "ugks_moments" in names and "ugks_residual" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _status_of(mesh, grid, gas, storage="f32", sweep="auto", raw_storage=None, block_velocities=0):
    lib = ugks.load()
    args = ugks._MeshArgs(mesh, grid)
    prm = ugks.make_params(gas, storage, sweep=sweep, block_velocities=block_velocities)
    if raw_storage is not None:
        prm.storage = raw_storage
    ctx = ctypes.c_void_p()
    st = lib.ugks_create(ctypes.byref(args.mesh), ctypes.byref(args.grid), ctypes.byref(prm), None, None,
                         ctypes.byref(ctx))
    assert not ctx.value
    return st, lib.ugks_last_error(None).decode()


def test_validation_errors_are_reported_before_any_device_work(lib):
    mesh = I.cavity_mesh(4)
    grid = I.midpoint_grid(6, -4, 4, 2)
    gas = I.Gas()
    bad = I.cavity_mesh(4)
    bad.face_neighbor = bad.face_neighbor.copy()
    bad.face_neighbor[0] = bad.face_owner[0]
    assert _status_of(bad, grid, gas)[0] == 2                        # UGKS_ERR_MESH
    bad = I.cavity_mesh(4)
    bad.cell_volume = bad.cell_volume.copy()
    bad.cell_volume[3] = -1.0
    assert _status_of(bad, grid, gas)[0] == 2
    bad = I.cavity_mesh(4)
    bad.face_normal = bad.face_normal * 2.0
    assert _status_of(bad, grid, gas)[0] == 2
    g2 = I.midpoint_grid(6, -4, 4, 2)
    g2.weight = g2.weight.copy()
    g2.weight[5] = -1.0
    assert _status_of(mesh, g2, gas)[0] == 3                         # UGKS_ERR_VGRID
    assert _status_of(mesh, grid, I.Gas(model="shakhov", Pr=2 / 3, K=1))[0] == 8   # UNSUPPORTED
    assert _status_of(mesh, grid, I.Gas(model="bgk", Pr=0.7))[0] == 1             # INVALID
    st, msg = _status_of(mesh, grid, gas, storage="f16", sweep="tiled")   # FP16 runs in the blocked sweep only
    assert st == 8 and "storage" in msg
    st, msg = _status_of(mesh, grid, gas, raw_storage=7)
    assert st == 1 and "storage" in msg
    st, msg = _status_of(mesh, grid, gas, block_velocities=256)          # compiled for 3-D, K_xi = 0 only
    assert st == 8 and "256" in msg
    st, msg = _status_of(mesh, grid, gas, block_velocities=96)
    assert st == 1 and "block_velocities" in msg
    out = ctypes.c_void_p()
    assert lib.ugks_create(None, None, None, None, None, ctypes.byref(out)) == 1
    assert lib.ugks_create(None, None, None, None, None, None) == 1
    assert lib.ugks_step(None, 1) == 1
    assert lib.ugks_destroy(None) == 0


def test_binding_raises_instead_of_falling_back(lib, monkeypatch):
    monkeypatch.setattr(ugks, "_lib", None)
    monkeypatch.setattr(ugks._build, "LIB", "/nonexistent/libugks.so")
    with pytest.raises(OSError):
        ugks.load(build_if_missing=False)


def test_warm_start_network_validates_its_arguments_on_the_host(lib):
    out = ctypes.c_void_p()
    assert lib.ugks_mlp_create(6, 9, 0, 6, 0, None, ctypes.byref(out)) == 1     # width 0
    assert "shape" in lib.ugks_mlp_last_error(None).decode()
    assert lib.ugks_mlp_create(6, 9, 64, 0, 0, None, ctypes.byref(out)) == 1    # no hidden layer
    assert lib.ugks_mlp_create(6, 9, 64, 2, 0, None, None) == 1                 # no output pointer
    assert not out.value
    assert lib.ugks_mlp_train(None, None, None, 1, 1, 1, ctypes.c_float(1e-3), 0, None) == 1
    assert lib.ugks_mlp_predict(None, None, 1, None) == 1
    assert lib.ugks_mlp_destroy(None) == 0


def test_declared_tensor_grid_is_checked_against_the_velocities(lib):
    """ugks_vgrid.tensor_n / axis declare a tensor-product grid (first axis
    fastest); a declaration that does not reproduce u is refused on the host."""
    mesh = I.cavity_mesh(4)
    gas = I.Gas()
    grid = I.midpoint_grid([32, 5], -4, 4, 2)
    assert grid.axes is not None
    wrong = I.VelocityGrid(u=grid.u, weight=grid.weight, axes=[grid.axes[1], grid.axes[0]])   # axes swapped
    st, msg = _status_of(mesh, wrong, gas)
    assert st == 3 and "tensor" in msg                                 # UGKS_ERR_VGRID
    shifted = I.VelocityGrid(u=grid.u, weight=grid.weight, axes=[grid.axes[0] + 1e-9, grid.axes[1]])
    st, msg = _status_of(mesh, shifted, gas)
    assert st == 3 and "match the axes" in msg
