"""The oracle against a separate slow transcription of the step (brute force).

tests/brute_ugks.py restates one UGKS step from the paper's equations and the
binding readings, with quadrature in place of every closed form the oracle
uses (Gaussian moments, half-range moments, the reduced Shakhov terms, the
derivatives of the interface Maxwellian, the time coefficients) and numpy
least squares in place of the oracle's explicit inverse.  On meshes of a few
cells and a few velocities, with every kind of boundary (diffuse wall with a
moving wall, far field, outflow), both models, K_xi = 0 .. 3, every limiter
and two regimes of dt / tau, two steps of both must agree to round-off
(1e-13 relative): a dropped term, a wrong sign, index or operand anywhere in
the oracle's step would not.  (Sec. 2.1, Eq. 3-42; Algorithm 5.)"""
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_2606_15720_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import brute_ugks as B  # noqa: E402


def strip1d():
    bcs = [I.BC(I.BC_FARFIELD, 1.15, (0.3, 0.0, 0.0), 1.2), I.BC(I.BC_OUTFLOW)]
    mesh = I.cartesian_mesh((4,), (0,), (1,), {"x-": 0, "x+": 1}, bcs)
    return mesh, I.midpoint_grid(8, -3.0, 3.0, 1), (0.1, 0.0, 0.0)


def box2d():
    bcs = [I.BC(I.BC_FARFIELD, 1.1, (0.3, 0.1, 0.0), 1.2), I.BC(I.BC_OUTFLOW),
           I.BC(I.BC_WALL, 1.0, (0.2, 0.0, 0.0), 1.3)]
    mesh = I.cartesian_mesh((3, 2), (0, 0), (1.0, 0.7), {"x-": 0, "x+": 1, "y-": 2, "y+": 2}, bcs)
    return mesh, I.midpoint_grid(3, -3.0, 3.0, 2), (0.2, 0.05, 0.0)


def tets3d():
    return I.box_tet_mesh(2, seed=7), I.midpoint_grid(2, -2.0, 2.0, 3), (0.2, 0.05, -0.1)


# (mesh builder, model, K, limiter)
CASES = {
    "strip1d_shakhov_Kxi2": (strip1d, "shakhov", 0, "venkatakrishnan"),
    "box2d_shakhov_wall_farfield_outflow": (box2d, "shakhov", 0, "venkatakrishnan"),
    "box2d_bgk_K2_barth_jespersen": (box2d, "bgk", 2, "barth_jespersen"),
    "box2d_shakhov_no_limiter": (box2d, "shakhov", 0, "none"),
    "tets3d_shakhov_venkatakrishnan": (tets3d, "shakhov", 0, "venkatakrishnan"),
    "tets3d_shakhov_barth_jespersen": (tets3d, "shakhov", 0, "barth_jespersen"),
    "tets3d_bgk_no_limiter": (tets3d, "bgk", 0, "none"),
    "tets3d_bgk_K2_venkatakrishnan": (tets3d, "bgk", 2, "venkatakrishnan"),
}
# (mu_ref, dt): dt / tau about 0.03 (collisionless-ish) and about 1
REGIMES = {"dt_small": (0.2, 0.01), "dt_tau": (0.01, 0.02)}


@pytest.mark.parametrize("regime", sorted(REGIMES))
@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_matches_the_brute_force_transcription(name, regime):
    build, model, K, limiter = CASES[name]
    mu_ref, dt = REGIMES[regime]
    mesh, grid, U0 = build()
    Pr = 2.0 / 3.0 if model == "shakhov" else 1.0
    gas = I.Gas(model=model, K=K, Pr=Pr, omega=0.81, mu_ref=mu_ref, cfl=0.8, limiter=limiter)
    prim = I.smooth_random_primitives(mesh, seed=4, amp=0.15, U0=U0)
    W0 = I.prim_to_conservative(prim, mesh.dim, K)
    f0 = O.initial_f(mesh, grid, W0, K)
    Wo, fo, _, _ = O.run(mesh, grid, gas, W0, f0, 2, dt=dt)
    bg = B.Gas(mesh.dim, K, model, Pr, gas.omega, mu_ref, gas.venkat_K, limiter)
    W1, f1 = B.step(mesh, grid.u, grid.weight, bg, W0, f0, dt)
    Wb, fb = B.step(mesh, grid.u, grid.weight, bg, W1, f1, dt)
    assert np.max(np.abs(Wb - W0)) > 1e-4 * np.max(np.abs(W0))     # the state did change
    for t in range(mesh.dim + 2):
        assert np.max(np.abs(Wb[:, t] - Wo[:, t])) <= 1e-13 * np.max(np.abs(Wo[:, t])), t
    for r in range(fo.shape[0]):
        assert np.max(np.abs(fb[r] - fo[r])) <= 1e-13 * np.max(np.abs(fo[r])), r


def test_brute_force_time_integrals_limits():
    """The transcription's own quadrature of c1 .. c5 against the limits of the
    time integrals (dt/tau -> 0: free transport; -> infinity: equilibrium)."""
    dt = 0.1
    g = B.time_integrals(dt, 1e9)
    assert g[0] == pytest.approx(dt, rel=1e-8) and g[1] == pytest.approx(-dt * dt / 2, rel=1e-8)
    assert abs(g[2]) < 1e-9 and abs(g[3]) < 1e-9 and abs(g[4]) < 1e-9
    g = B.time_integrals(dt, 1e-6)
    assert g[2] == pytest.approx(dt, rel=1e-4) and abs(g[0]) < 1e-5
