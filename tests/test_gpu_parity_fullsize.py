"""Full-size parity: the 3-D sphere workload (~1e5 tetrahedra x 32^3
velocities, Shakhov, FP32 storage) in the launch configuration the benchmark
times.  The oracle cannot step 3.3e9 phase-space points, so it recomputes
sampled cells one by one: a cell's W^{n+1} and f^{n+1} depend only on cells
within two face hops (gradients of the face neighbours, their macroscopic
slopes, their heat fluxes), so the oracle steps the 3-ring patch around the
samples, closed by outflow faces, with the device's time step."""
import numpy as np
import pytest

import oracle as O
from paper_2606_15720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_sphere_full_size_sampled_cells_match_oracle():
    from paper_2606_15720_gb300 import ugks as U
    mesh = I.sphere_tet_mesh(100_000, seed=2)
    grid = I.midpoint_grid(32, -12, 12, 3)
    gas = I.Gas(model="shakhov", Pr=2 / 3, omega=0.81, mu_ref=I.mu_ref_from_kn(0.05, 0.81), cfl=0.8)
    u_inf = mesh.bc[1].u[0]
    prim = I.smooth_random_primitives(mesh, seed=9, amp=0.1, U0=(u_inf, 0, 0), length=(12, 10, 10))
    W0 = I.prim_to_conservative(prim, 3, 0)
    rng = np.random.default_rng(1234)
    picks = []
    for b in range(3):   # wall, far field, outflow
        owners = mesh.face_owner[mesh.face_neighbor == -(b + 1)]
        picks += list(rng.choice(owners, size=2, replace=False))
    picks += list(rng.choice(mesh.n_cells, size=3, replace=False))
    picks = np.array(sorted(set(int(c) for c in picks)), dtype=np.int64)
    with U.Solver(mesh, grid, gas, W0, storage="f32") as s:
        dt = s.dt
        s.step(1)
        W1 = s.moments()
        f1 = s.get_f(picks)                                   # [n, 1, nv]
    cells, pm = I.submesh(mesh, picks, rings=3)
    f0 = O.initial_f(pm, grid, W0[cells], 0)
    Wo, fo, _, _ = O.run(pm, grid, gas, W0[cells], f0, 1, dt=dt)
    loc = np.searchsorted(cells, picks)
    for s_, c in enumerate(picks):
        Wg, Wr = W1[c], Wo[loc[s_]]
        err = np.max(np.abs(Wg - Wr)) / np.max(np.abs(Wr))
        assert err <= 1e-5, (int(c), err, Wg, Wr)
        ferr = np.max(np.abs(f1[s_, 0] - fo[0, loc[s_]])) / np.max(np.abs(fo[0, loc[s_]]))
        assert ferr <= 1e-5, (int(c), ferr)
