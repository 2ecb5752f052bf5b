"""Host logic of the warm-start driver (paper_2606_15720_gb300/warmstart.py),
without a GPU: case construction, the convergence loop, the error measure."""
import math

import numpy as np

from paper_2606_15720_gb300 import inputs as I
from paper_2606_15720_gb300 import warmstart as WS


class FakeSolver:
    """Residual r0 q^n after n steps (geometric decay), no device."""

    def __init__(self, r0, q):
        self.r0, self.q, self.n = r0, q, 0

    def step(self, n):
        self.n += n

    def residual(self):
        return np.array([self.r0 * self.q ** self.n, 0.0, 0.0, 0.0])


def test_converge_reports_the_first_check_below_the_tolerance():
    a, b = FakeSolver(1e-3, 0.999), FakeSolver(1e-3, 0.995)
    steps = WS.converge([a, b], tol=1e-6, max_steps=20_000, check_every=100)
    # 1e-3 q^n < 1e-6  <=>  n > 3 ln 10 / -ln q, rounded up to the next check
    for s, q in zip(steps, (0.999, 0.995)):
        n = 3 * math.log(10) / -math.log(q)
        assert s == 100 * math.ceil(n / 100)


def test_converge_gives_none_when_the_step_budget_runs_out():
    s = FakeSolver(1.0, 0.9999)
    assert WS.converge([s], tol=1e-6, max_steps=1000, check_every=100) == [None]


class FailingSolver(FakeSolver):
    """Raises the library's non-physical error from step ``fail_at`` on."""

    def __init__(self, fail_at):
        super().__init__(1.0, 1.0)
        self.fail_at = fail_at

    def residual(self):
        from paper_2606_15720_gb300 import ugks as U
        if self.n >= self.fail_at:
            raise U.UGKSError(6, "non-physical state")
        return super().residual()


def test_converge_stops_stepping_a_case_that_became_non_physical():
    ok, bad = FakeSolver(1e-3, 0.995), FailingSolver(300)
    steps = WS.converge([ok, bad], tol=1e-6, max_steps=20_000, check_every=100)
    assert steps[0] == 100 * math.ceil(3 * math.log(10) / -math.log(0.995) / 100)
    assert steps[1] is None
    assert bad.n == 300                       # not stepped after its failure was seen


def test_batch_family_cases_use_the_batch_workload_recipe():
    mesh, grid, gas, W0 = WS.cylinder_case(6.0, 0.05, 400, None, seed=3, family="batch")
    assert gas.model == "bgk" and gas.venkat_K == 1.0
    u_inf = 6.0 * math.sqrt(5.0 / 6.0)
    vmax = max(u_inf + 4.0, 3.5 * math.sqrt(1.0 + 36.0 / 3.0))
    n = int(round(math.sqrt(grid.n_v)))
    assert n == min(48, max(20, math.ceil(2 * vmax / 0.7)))
    np.testing.assert_allclose(W0, I.prim_to_conservative(I.cylinder_potential_primitives(mesh, u_inf), 2, 0))
    nb = mesh.face_neighbor
    yc = mesh.face_centroid[nb < 0, 1]
    assert np.all(-(nb[nb < 0][np.abs(np.abs(yc) - 5.0) < 1e-9] + 1) == 2)     # outflow lateral edges
    mesh_s, _, gas_s, _ = WS.cylinder_case(2.0, 0.1, 400, 24, seed=3)
    nb = mesh_s.face_neighbor
    yc = mesh_s.face_centroid[nb < 0, 1]
    assert gas_s.model == "shakhov"
    assert np.all(-(nb[nb < 0][np.abs(np.abs(yc) - 5.0) < 1e-9] + 1) == 1)   # far-field lateral edges


def test_rel_linf_is_per_field_and_relative_to_the_reference_magnitude():
    ref = np.array([[1.0, -2.0], [0.5, 4.0]])
    w = ref + np.array([[0.1, 0.0], [0.0, -0.2]])
    np.testing.assert_allclose(WS.rel_linf(w, ref), [0.1, 0.05])


def test_cylinder_cases_resolve_the_free_stream_and_start_from_it():
    for mach in (1.5, 3.0):
        mesh, grid, gas, W0 = WS.cylinder_case(mach, 0.1, 400, 28, seed=1)
        fs = WS.freestream_fields(mesh)
        assert fs[0] == 1.0 and fs[-1] == 1.0
        assert fs[1] == mesh.bc[1].u[0] and fs[2] == 0.0
        # velocity range covers the free stream and the stagnation temperature
        vmax = np.abs(grid.u).max()
        assert vmax >= fs[1] + 3.5 and vmax >= 3.0 * math.sqrt(1.0 + mach * mach / 3.0)
        # the start is the free stream everywhere
        prim = I.uniform_primitives(mesh, 1.0, mesh.bc[1].u, 1.0)
        np.testing.assert_allclose(W0, I.prim_to_conservative(prim, 2, 0))
        assert gas.model == "shakhov" and gas.K == 0
