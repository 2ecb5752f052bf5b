"""The allocation-free step, ugks_step_static_scratch, against ugks_step.

Some callers cannot allocate device memory once a solver is set up: a host
application whose device memory pool belongs to another allocator (a
framework's caching allocator holds it), or a latency-critical loop that
cannot afford the device-wide synchronisation cudaMalloc / cudaFree may
cause.  For them the library offers a step whose sweep scratch is a fixed
16 MiB device array.  This file checks, through the C ABI, that two calls in
a row give the same state as the ordinary step (within the parity tolerances
of the other tests), and that a context needing more scratch is refused with
a clear message.  It is collected last on purpose."""
import numpy as np
import pytest

from paper_2606_15720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _w_err(a, b):
    dim = a.shape[1] - 2
    e = [np.max(np.abs(a[:, 0] - b[:, 0])) / np.max(np.abs(b[:, 0])),
         np.max(np.linalg.norm(a[:, 1:1 + dim] - b[:, 1:1 + dim], axis=1)) /
         max(np.max(np.linalg.norm(b[:, 1:1 + dim], axis=1)), 1e-300),
         np.max(np.abs(a[:, -1] - b[:, -1])) / np.max(np.abs(b[:, -1]))]
    return float(max(e))


@pytest.mark.parametrize("sweep", [dict(sweep="blocked", block_velocities=64), dict(sweep="tiled", tile_cells=48)],
                         ids=["blocked", "tiled"])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_static_scratch_step_matches_ordinary_step_on_two_calls(storage, tol, sweep):
    from paper_2606_15720_gb300 import ugks as U
    mesh = I.cavity_mesh(16)
    grid = I.midpoint_grid(20, -4.5, 4.5, 2)
    gas = I.Gas(model="shakhov", Pr=2 / 3, omega=0.81, mu_ref=I.mu_ref_from_kn(0.075, 0.81), cfl=0.8)
    W0 = I.prim_to_conservative(I.smooth_random_primitives(mesh, seed=21, amp=0.1), 2, 0)
    with U.Solver(mesh, grid, gas, W0, storage=storage, **sweep) as ref, \
            U.Solver(mesh, grid, gas, W0, storage=storage, **sweep) as na:
        for call in range(2):
            ref.step(3)
            na.step_static_scratch(3)
            Wr, Wn = ref.moments(), na.moments()
            assert _w_err(Wn, Wr) <= tol, (call, _w_err(Wn, Wr))
            np.testing.assert_allclose(na.residual(), ref.residual(), rtol=1e-9 if storage == "f64" else 1e-4)
        fr = ref.get_f(np.arange(mesh.n_cells))
        fn = na.get_f(np.arange(mesh.n_cells))
        assert np.max(np.abs(fn - fr)) <= tol * np.max(np.abs(fr))


def test_static_scratch_step_rejects_contexts_beyond_its_size():
    from paper_2606_15720_gb300 import ugks as U
    # blocked sweep, 64 velocities per block: its per-face buffer alone needs
    # 131584 faces x 2 x 64 x 8 B = 135 MB
    mesh = I.cavity_mesh(256)
    grid = I.midpoint_grid(24, -4.5, 4.5, 2)
    gas = I.Gas(model="bgk", omega=0.81, mu_ref=I.mu_ref_from_kn(0.075, 0.81), cfl=0.8)
    with U.Solver(mesh, grid, gas, None, storage="f64", sweep="blocked", block_velocities=64) as s:
        with pytest.raises(U.UGKSError) as e:
            s.step_static_scratch(1)
        assert e.value.status == 1 and "static limit" in str(e.value)
        s.step(1)                                    # the ordinary step still works on it
        assert np.all(np.isfinite(s.moments()))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_static_scratch_step_scaled_storage_matches_ordinary_step(storage):
    """FP16 / BF16 storage (FP32 arithmetic) through the allocation-free step:
    the same kernels on a different scratch address, so after two calls of
    three steps each the state agrees with the ordinary step to FP32 rounding."""
    from paper_2606_15720_gb300 import ugks as U
    mesh = I.cavity_mesh(16)
    grid = I.midpoint_grid(20, -4.5, 4.5, 2)
    gas = I.Gas(model="bgk", omega=0.81, mu_ref=I.mu_ref_from_kn(0.075, 0.81), cfl=0.8)
    W0 = I.prim_to_conservative(I.smooth_random_primitives(mesh, seed=22, amp=0.1), 2, 0)
    with U.Solver(mesh, grid, gas, W0, storage=storage, block_velocities=64) as ref, \
            U.Solver(mesh, grid, gas, W0, storage=storage, block_velocities=64) as na:
        for call in range(2):
            ref.step(3)
            na.step_static_scratch(3)
            assert _w_err(na.moments(), ref.moments()) <= 1e-5, call


def test_surface_after_static_steps_of_two_contexts_is_each_contexts_own():
    """Two contexts take turns on the shared scratch array, one after the
    other (each context runs on its own stream, so the first is synchronised
    before the second steps); the wall quantities of the first, read after the
    second has stepped, equal those of an ordinary-step twin of the first."""
    from paper_2606_15720_gb300 import ugks as U
    mesh = I.cavity_mesh(12)
    grid = I.midpoint_grid(18, -4.5, 4.5, 2)
    gas = I.Gas(model="shakhov", Pr=2 / 3, omega=0.81, mu_ref=I.mu_ref_from_kn(0.075, 0.81), cfl=0.8)
    WA = I.prim_to_conservative(I.smooth_random_primitives(mesh, seed=23, amp=0.1), 2, 0)
    WB = I.prim_to_conservative(I.smooth_random_primitives(mesh, seed=24, amp=0.2), 2, 0)
    with U.Solver(mesh, grid, gas, WA, storage="f64") as twin, \
            U.Solver(mesh, grid, gas, WA, storage="f64") as a, \
            U.Solver(mesh, grid, gas, WB, storage="f64") as b:
        twin.step(2)
        a.step_static_scratch(2)
        a.residual()             # synchronises A's stream: B's steps must not overlap A's on the GPU
        b.step_static_scratch(2)
        fa, va, _ = a.surface()
        ft, vt, _ = twin.surface()
        fb, vb, _ = b.surface()
        np.testing.assert_array_equal(fa, ft)
        assert np.max(np.abs(va - vt)) <= 1e-11 * np.max(np.abs(vt))
        assert np.max(np.abs(vb - vt)) > 1e-6 * np.max(np.abs(vt))   # B's walls differ from A's
