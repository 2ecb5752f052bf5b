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
