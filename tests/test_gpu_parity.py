"""Parity of the CUDA path with the FP64 oracle, element by element.

Every case builds seeded synthetic inputs, runs the CUDA library through the
C ABI (ugks_create / ugks_step / ugks_moments / ugks_get_f) and the oracle on
the same inputs, and compares W and the distributions.  Tolerances:
  * FP64 storage: relative L-inf <= 1e-11 on W and f (round-off only);
  * FP32 storage: relative L-inf on W <= 1e-5 after one step and <= 1e-4
    after 100 steps; f <= 1e-5 after one step.
Relative L-inf of W: density and energy each as max_i |a_i - b_i| / max_i |b_i|;
momentum as a vector, max_i |a_i - b_i|_2 / max_i |b_i|_2 (its transverse
components can be near zero, so they are measured against the momentum
scale); the largest of the three.  For f: per reduced distribution."""
import numpy as np
import pytest

import oracle as O
from paper_2606_15720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2606_15720_gb300 import ugks
    ugks.load()
    return ugks


def rel_linf(a, b, axis_fields=-1):
    a = np.asarray(a)
    b = np.asarray(b)
    if axis_fields is None:
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
    a2 = np.moveaxis(a, axis_fields, 0).reshape(a.shape[axis_fields], -1)
    b2 = np.moveaxis(b, axis_fields, 0).reshape(b.shape[axis_fields], -1)
    out = 0.0
    for x, y in zip(a2, b2):
        scale = np.max(np.abs(y))
        if scale == 0.0:
            scale = 1.0
        out = max(out, float(np.max(np.abs(x - y)) / scale))
    return out


def w_err(a, b):
    """Relative L-inf error of conservative fields [n, dim+2] (density, momentum vector, energy)."""
    a = np.asarray(a)
    b = np.asarray(b)
    dim = a.shape[1] - 2
    e_rho = np.max(np.abs(a[:, 0] - b[:, 0])) / np.max(np.abs(b[:, 0]))
    mom = np.max(np.linalg.norm(b[:, 1:1 + dim], axis=1))
    e_mom = np.max(np.linalg.norm(a[:, 1:1 + dim] - b[:, 1:1 + dim], axis=1)) / (mom if mom > 0 else 1.0)
    e_E = np.max(np.abs(a[:, -1] - b[:, -1])) / np.max(np.abs(b[:, -1]))
    return float(max(e_rho, e_mom, e_E))


# device organisations of the sweep: the blocked sweep with 32, 64, 128 and
# (3-D, one reduced distribution) 256 velocities per block, its fused form
# (each cell evaluates its faces' fluxes in the first-stage kernel), and the
# tiled sweep (small tiles: several per CTA)
SWEEPS = {
    "blocked64": dict(sweep="blocked", block_velocities=64),
    "blocked32": dict(sweep="blocked", block_velocities=32),
    "blocked128": dict(sweep="blocked", block_velocities=128),
    "blocked256": dict(sweep="blocked", block_velocities=256),
    "blocked_fused64": dict(sweep="blocked_fused", block_velocities=64),   # fluxes evaluated per cell with stage 1
    "tiled": dict(sweep="tiled", tile_cells=48),
    "scaled": dict(sweep="blocked"),   # the storage argument selects FP16 / BF16
    "scaled_fused": dict(sweep="blocked_fused"),
}
_oracle_cache = {}


def supports(sweep, mesh, gas):
    """256 velocities per block are compiled for 3-D with K_xi = 0 only."""
    return sweep != "blocked256" or (mesh.dim == 3 and gas.K == 0)


def run_pair(U, mesh, grid, gas, prim, nsteps, storage, sweep="blocked64", key=None):
    if not supports(sweep, mesh, gas):
        pytest.skip("256 velocities per block: 3-D with K_xi = 0 only")
    W0 = I.prim_to_conservative(prim, mesh.dim, gas.K)
    with U.Solver(mesh, grid, gas, W0, storage=storage, **SWEEPS[sweep]) as s:
        dt = s.dt
        s.step(nsteps)
        Wg = s.moments()
        fg = s.get_f(np.arange(mesh.n_cells))            # [cell, r, k]
        res = s.residual()
    ck = None if key is None else (key, nsteps, dt)
    if ck in _oracle_cache:
        Wo, fo, dto, diag = _oracle_cache[ck]
    else:
        f0 = O.initial_f(mesh, grid, W0, gas.K)
        Wo, fo, dto, diag = O.run(mesh, grid, gas, W0, f0, nsteps, dt=dt)
        if ck is not None:
            _oracle_cache[ck] = (Wo, fo, dto, diag)
    return Wg, np.transpose(fg, (1, 0, 2)), res, Wo, fo, diag, dt, dto


# ---------------------------------------------------------------------------
# case builders (small sizes that still span several tiles and a ragged tail)
# ---------------------------------------------------------------------------

def cavity_case(n=16, nvx=20, model="bgk"):
    mesh = I.cavity_mesh(n)
    grid = I.midpoint_grid(nvx, -4.5, 4.5, 2)        # 400 velocities: 12 full blocks + a ragged tail
    gas = I.Gas(model=model, Pr=1.0 if model == "bgk" else 2 / 3, omega=0.81,
                mu_ref=I.mu_ref_from_kn(0.075, 0.81), cfl=0.8)
    prim = I.smooth_random_primitives(mesh, seed=11, amp=0.1)
    return mesh, grid, gas, prim


def periodic3d_case(model="shakhov", K=0):
    mesh = I.periodic_box((5, 4, 3))
    grid = I.midpoint_grid(7, -5, 5, 3)              # 343 velocities
    gas = I.Gas(model=model, K=K, Pr=2 / 3 if model == "shakhov" else 1.0, mu_ref=0.02, omega=0.72)
    prim = I.smooth_random_primitives(mesh, seed=5, amp=0.15, U0=(0.3, -0.1, 0.2))
    return mesh, grid, gas, prim


def strip1d_case():
    mesh = I.cartesian_mesh((40,), (0,), (1,), {"x-": 0, "x+": 1},
                            [I.BC(I.BC_FARFIELD, 1.0, (0.2, 0, 0), 1.0), I.BC(I.BC_OUTFLOW)])
    grid = I.midpoint_grid(45, -8, 8, 1)
    gas = I.Gas(model="shakhov", Pr=2 / 3, mu_ref=0.01, omega=0.5, shock_tau_fix=True)
    prim = I.uniform_primitives(mesh)
    x = mesh.cell_centroid[:, 0]
    prim[:, 0] = np.where(x < 0.5, 1.0, 0.3)
    prim[:, -1] = np.where(x < 0.5, 1.5, 1.0)
    return mesh, grid, gas, prim


def wheel_mesh(n=10, radii=(0.5, 1.0, 1.6, 2.4)):
    """2-D polygonal mesh: a regular n-gon at the centre (n faces, more than
    the 8 of the pipelined kernels' incidence table) inside rings of n quads
    each; far-field outer edge.  Built here, face by face (shoelace areas and
    centroids), for the kernels that such cells take."""
    th = 2 * np.pi * (np.arange(n) + 0.25) / n
    pts = [np.stack([r * np.cos(th), r * np.sin(th)], 1) for r in radii]
    cells = [pts[0]]                                    # the n-gon
    for k in range(len(radii) - 1):
        for i in range(n):
            j = (i + 1) % n
            cells.append(np.array([pts[k][i], pts[k + 1][i], pts[k + 1][j], pts[k][j]]))

    def area_centroid(P):
        x, y = P[:, 0], P[:, 1]
        xn, yn = np.roll(x, -1), np.roll(y, -1)
        cr = x * yn - xn * y
        A = 0.5 * cr.sum()
        return abs(A), np.array([((x + xn) * cr).sum(), ((y + yn) * cr).sum()]) / (6 * A)

    vol, cen = zip(*(area_centroid(P) for P in cells))
    edges = {}
    for c, P in enumerate(cells):
        for a in range(len(P)):
            key = tuple(sorted((tuple(np.round(P[a], 12)), tuple(np.round(P[(a + 1) % len(P)], 12)))))
            edges.setdefault(key, []).append(c)
    own, nei, area, nrm, fcen = [], [], [], [], []
    for (pa, pb), cs in edges.items():
        pa, pb = np.array(pa), np.array(pb)
        mid = 0.5 * (pa + pb)
        t = pb - pa
        nv = np.array([t[1], -t[0]]) / np.linalg.norm(t)
        o = cs[0]
        if np.dot(nv, mid - cen[o]) < 0:
            nv = -nv
        own.append(o)
        nei.append(cs[1] if len(cs) == 2 else -1)
        area.append(np.linalg.norm(t))
        nrm.append(nv)
        fcen.append(mid)
    nf = len(own)
    return I.Mesh(dim=2, cell_volume=np.array(vol), cell_centroid=np.array(cen),
                  face_owner=np.array(own, dtype=np.int64), face_neighbor=np.array(nei, dtype=np.int64),
                  face_area=np.array(area), face_normal=np.array(nrm), face_centroid=np.array(fcen),
                  face_shift=np.zeros((nf, 2)), bc=[I.BC(I.BC_FARFIELD, 1.0, (0.3, 0.1, 0.0), 1.1)],
                  name=f"wheel{n}")


def wheel_case():
    mesh = wheel_mesh()
    grid = I.midpoint_grid(14, -5, 5, 2)                # 196 velocities: 6 blocks of 32 + a ragged tail
    gas = I.Gas(model="shakhov", Pr=2 / 3, omega=0.81, mu_ref=0.05, cfl=0.8)
    prim = I.smooth_random_primitives(mesh, seed=6, amp=0.1, U0=(0.3, 0.1, 0.0), length=(5, 5))
    return mesh, grid, gas, prim


def sphere_case(cells=2500, nvx=11, mach=2.0, vmax=6.0):
    # the velocity grid must resolve the gas (spacing ~ thermal speed): 11^3 on [-6, 6]^3
    mesh = I.sphere_tet_mesh(cells, seed=3, mach=mach)
    u_inf = mesh.bc[1].u[0]
    grid = I.midpoint_grid(nvx, -vmax, vmax, 3)
    gas = I.Gas(model="shakhov", Pr=2 / 3, omega=0.81, mu_ref=I.mu_ref_from_kn(0.05, 0.81), cfl=0.8)
    prim = I.smooth_random_primitives(mesh, seed=9, amp=0.1, U0=(u_inf, 0, 0), length=(12, 10, 10))
    return mesh, grid, gas, prim


def cylinder_case(cells=1500, nvx=13):
    mesh = I.cylinder_tri_mesh(cells, seed=4, mach=3.0)
    u_inf = mesh.bc[1].u[0]
    grid = I.midpoint_grid(nvx, -9, 9, 2)
    gas = I.Gas(model="bgk", omega=0.81, mu_ref=I.mu_ref_from_kn(0.1, 0.81), cfl=0.8, K=2)
    prim = I.smooth_random_primitives(mesh, seed=2, amp=0.1, U0=(u_inf, 0, 0), length=(12, 10))
    return mesh, grid, gas, prim


def tensor_cases():
    """Velocity grids whose fastest axis has 32 points (every row of 32
    velocities is one line along that axis): the separable path of the
    kernels.  2-D cavity (32 x 20), 3-D sphere (32 x 10 x 10, Shakhov),
    3-D periodic box with two reduced distributions (32 x 6 x 6, BGK K = 2),
    1-D strip (32 points, one row)."""
    def cavity():
        mesh, _, gas, prim = cavity_case(model="shakhov")
        return mesh, I.midpoint_grid([32, 20], -4.5, 4.5, 2), gas, prim

    def sphere():
        mesh, _, gas, prim = sphere_case()
        return mesh, I.midpoint_grid([32, 10, 10], -6.0, 6.0, 3), gas, prim

    def periodic():
        mesh, _, gas, prim = periodic3d_case("bgk", K=2)
        return mesh, I.midpoint_grid([32, 6, 6], -5, 5, 3), gas, prim

    def strip():
        mesh, _, gas, prim = strip1d_case()
        return mesh, I.midpoint_grid(32, -8, 8, 1), gas, prim
    return {"cavity_tensor32": cavity, "sphere_tensor32": sphere, "periodic3d_tensor32_K2": periodic,
            "strip1d_tensor32": strip}


CASES = {
    "cavity_bgk": cavity_case,
    "cavity_shakhov": lambda: cavity_case(model="shakhov"),
    "periodic3d_shakhov": periodic3d_case,
    "periodic3d_bgk_K2": lambda: periodic3d_case("bgk", K=2),
    "strip1d_farfield_outflow": strip1d_case,
    "sphere_tet": sphere_case,
    "cylinder_tri_K2": cylinder_case,
    **tensor_cases(),
}


@pytest.mark.parametrize("sweep", sorted(k for k in SWEEPS if not k.startswith("scaled")))
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_matches_oracle(U, name, sweep):
    mesh, grid, gas, prim = CASES[name]()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 3, "f64", sweep, key=name)
    assert w_err(Wg, Wo) <= 1e-11, w_err(Wg, Wo)
    assert rel_linf(fg, fo, axis_fields=0) <= 1e-11
    np.testing.assert_allclose(res, diag[-1, :mesh.dim + 2], rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("sweep", sorted(k for k in SWEEPS if not k.startswith("scaled")))
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_one_step_matches_oracle(U, name, sweep):
    mesh, grid, gas, prim = CASES[name]()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 1, "f32", sweep, key=name)
    assert w_err(Wg, Wo) <= 1e-5, w_err(Wg, Wo)
    assert rel_linf(fg, fo, axis_fields=0) <= 1e-5, rel_linf(fg, fo, axis_fields=0)


LONG_CASES = {
    "cavity_bgk": cavity_case,
    "periodic3d_shakhov": periodic3d_case,
    "sphere_tet_small": lambda: sphere_case(cells=1200, nvx=12),
    "sphere_tensor32_small": lambda: (lambda c: (c[0], I.midpoint_grid([32, 8, 8], -6.0, 6.0, 3), c[2], c[3]))(
        sphere_case(cells=1200, nvx=12)),
}


@pytest.mark.parametrize("sweep", ["blocked64", "blocked256", "tiled"])
@pytest.mark.parametrize("name", sorted(LONG_CASES))
def test_fp32_hundred_steps_matches_oracle(U, name, sweep):
    mesh, grid, gas, prim = LONG_CASES[name]()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 100, "f32", sweep, key="long_" + name)
    assert w_err(Wg, Wo) <= 1e-4, w_err(Wg, Wo)


def sphere_benchmark_physics_case():
    """The benchmark's physics on a reduced mesh: Ma 5 impulsive freestream
    start (Kn 0.05, Shakhov, Pr 2/3, diffuse wall at the stagnation
    temperature, far field, outflow) on 1200 tetrahedra of the same
    generator, velocities on [-12, 12]^3 with 32 points along the flow axis
    (the tensor-row path) and 20 across."""
    mesh = I.sphere_tet_mesh(1200, seed=2)
    grid = I.midpoint_grid([32, 20, 20], -12.0, 12.0, 3)
    gas = I.Gas(model="shakhov", K=0, Pr=2.0 / 3.0, omega=0.81, mu_ref=I.mu_ref_from_kn(0.05, 0.81), cfl=0.8)
    prim = I.uniform_primitives(mesh, 1.0, mesh.bc[1].u, 1.0)
    return mesh, grid, gas, prim


@pytest.mark.parametrize("sweep", ["blocked64", "blocked256"])
def test_fp32_hundred_steps_at_benchmark_physics(U, sweep):
    """100 FP32 steps of the Ma 5 sphere on [-12, 12]^3 against the FP64
    oracle: W within the FP32 bound of 1e-4 after 100 steps."""
    mesh, grid, gas, prim = sphere_benchmark_physics_case()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 100, "f32", sweep, key="ma5_sphere")
    assert np.all(np.isfinite(Wg))
    assert w_err(Wg, Wo) <= 1e-4, w_err(Wg, Wo)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_scaled_storage_hundred_steps_at_benchmark_physics(U, storage):
    """100 steps of the Ma 5 sphere with FP16 / BF16 storage: each step rounds
    every stored value to eps of its deviation from the reference Maxwellian
    (at most 0.1 of max |f| here), which moves W by at most that much per step
    (CFL < 1); accumulated linearly over 100 steps: W within 100 eps 0.1."""
    mesh, grid, gas, prim = sphere_benchmark_physics_case()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 100, storage, "scaled", key="ma5_sphere")
    assert w_err(Wg, Wo) <= 100 * STORAGE_EPS[storage] * 0.1, w_err(Wg, Wo)


def cylinder_hypersonic_case(mach=7.5, kn=0.005, cells=1500):
    """The upper end of the cylinder batch workload, reduced: Ma 7.5,
    Kn 0.005, BGK with K_v = 1, diffuse wall at the stagnation temperature,
    the potential-flow start, 45^2 velocities of spacing 0.7 on
    [-15.6, 15.6]^2 (the batch's grid rule), 1500 triangles."""
    mesh = I.cylinder_tri_mesh(cells, seed=11, mach=mach)
    u_inf = mesh.bc[1].u[0]
    vmax = max(u_inf + 4.0, 3.5 * np.sqrt(1.0 + mach * mach / 3.0))
    nvx = int(min(48, max(20, np.ceil(2.0 * vmax / 0.7))))
    grid = I.midpoint_grid(nvx, -vmax, vmax, 2)
    gas = I.Gas(model="bgk", K=0, Pr=1.0, omega=0.81, mu_ref=I.mu_ref_from_kn(kn, 0.81), cfl=0.8, venkat_K=1.0)
    return mesh, grid, gas, I.cylinder_potential_primitives(mesh, u_inf)


@pytest.mark.parametrize("storage,bound", [("f64", 1e-11), ("f32", 1e-4)])
def test_hypersonic_cylinder_hundred_steps(U, storage, bound):
    """100 steps of the Ma 7.5 cylinder against the FP64 oracle: FP64 to
    round-off, FP32 within 1e-4 (the FP32 bound after 100 steps); the wake's density falls
    below 1e-2 of the free stream and stays positive."""
    mesh, grid, gas, prim = cylinder_hypersonic_case()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 100, storage, "blocked128", key="ma75_cylinder")
    assert w_err(Wg, Wo) <= bound, w_err(Wg, Wo)
    assert np.min(Wo[:, 0]) > 0.0 and np.min(Wo[:, 0]) < 0.05


@pytest.mark.parametrize("storage,steps,bound", [("f64", 3, 1e-11), ("f32", 1, 1e-5)])
def test_cells_with_more_than_eight_faces(U, storage, steps, bound):
    """A ten-sided cell sends the reconstruction and first stage to their
    non-pipelined kernels: W and f against the oracle (FP64 to round-off,
    FP32 within the one-step bound).  Scaled FP16 storage, which needs the
    pipelined kernels, is refused."""
    mesh, grid, gas, prim = wheel_case()
    assert mesh.closure_residual() < 1e-13
    assert np.max(np.bincount(np.concatenate([mesh.face_owner, mesh.face_neighbor[mesh.face_neighbor >= 0]]))) == 10
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, steps, storage, "blocked64")
    assert w_err(Wg, Wo) <= bound, w_err(Wg, Wo)
    for r in range(fo.shape[0]):
        assert rel_linf(fg[r], fo[r], None) <= bound
    with pytest.raises(U.UGKSError):
        U.Solver(mesh, grid, gas, I.prim_to_conservative(prim, 2, gas.K), storage="f16")


def test_cavity_config_200_steps_fp64(U):
    """32x32 cavity, 24x24 grid, Kn 0.075, FP64, 200 steps (the correctness workload)."""
    mesh = I.cavity_mesh(32)
    grid = I.midpoint_grid(24, -4.5, 4.5, 2)
    gas = I.Gas(model="bgk", omega=0.81, mu_ref=I.mu_ref_from_kn(0.075, 0.81), cfl=0.8)
    prim = I.uniform_primitives(mesh)
    Wg, fg, res, Wo, fo, diag, dt, dto = run_pair(U, mesh, grid, gas, prim, 200, "f64")
    assert w_err(Wg, Wo) <= 1e-10
    assert abs(dt - O.time_step(mesh, grid, 0.8)) <= 1e-15 * dt
    # the lid drives the gas and the walls hold the mass
    assert np.max(Wg[:, 1]) > 1e-3
    assert mesh.cell_volume @ Wg[:, 0] == pytest.approx(1.0, rel=1e-12)


def test_tiling_does_not_change_the_result(U):
    """Faces shared by tiles are evaluated identically by both: W of the tiled
    sweep is bitwise independent of the tile size (FP64 and FP32)."""
    mesh, grid, gas, prim = sphere_case(cells=2000, nvx=9)
    W0 = I.prim_to_conservative(prim, 3, 0)
    for storage in ("f64", "f32"):
        outs = []
        for tc in (16, 40, 0):
            with U.Solver(mesh, grid, gas, W0, storage=storage, tile_cells=tc, sweep="tiled") as s:
                s.step(4)
                outs.append(s.moments())
        assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_sweep_organisations_agree(U):
    """The blocked sweep at 32, 64, 128 and 256 velocities per block and the
    tiled sweep compute the same step: FP64 W agrees to round-off."""
    mesh, grid, gas, prim = sphere_case(cells=2000, nvx=9)
    W0 = I.prim_to_conservative(prim, 3, 0)
    outs = {}
    for name, kw in SWEEPS.items():
        if name == "scaled":
            continue
        with U.Solver(mesh, grid, gas, W0, storage="f64", **kw) as s:
            s.step(4)
            outs[name] = s.moments()
    for name in outs:
        assert w_err(outs[name], outs["tiled"]) <= 1e-13, name


@pytest.mark.parametrize("sweep", ["blocked64", "tiled"])
def test_conservation_on_periodic_box_fp32(U, sweep):
    mesh, grid, gas, prim = periodic3d_case()
    W0 = I.prim_to_conservative(prim, 3, 0)
    kw = dict(SWEEPS[sweep])
    if sweep == "tiled":
        kw["tile_cells"] = 8
    with U.Solver(mesh, grid, gas, W0, storage="f32", **kw) as s:
        s.step(20)
        W = s.moments()
    tot0, tot = mesh.cell_volume @ W0, mesh.cell_volume @ W
    np.testing.assert_allclose(tot, tot0, rtol=1e-13, atol=1e-13)


def test_zero_steps_and_checkpoint_roundtrip(U):
    mesh, grid, gas, prim = cavity_case(n=8, nvx=10)
    W0 = I.prim_to_conservative(prim, 2, 0)
    with U.Solver(mesh, grid, gas, W0, storage="f64") as s:
        s.step(0)
        np.testing.assert_array_equal(s.moments(), W0)
        np.testing.assert_array_equal(s.residual(), 0.0)
        s.step(3)
        W3, f3, k = s.get_state()
        assert k == 3
        s.step(4)
        W7 = s.moments()
    with U.Solver(mesh, grid, gas, W0, storage="f64") as s2:
        s2.set_state(W3, f3, 3)
        s2.step(4)
        assert np.array_equal(s2.moments(), W7)


def test_solve_one_shot_with_host_buffers(U):
    mesh, grid, gas, prim = cavity_case(n=8, nvx=10)
    W0 = I.prim_to_conservative(prim, 2, 0)
    Wout, res = U.solve(mesh, grid, gas, W0, 5, storage="f64")
    f0 = O.initial_f(mesh, grid, W0, 0)
    with U.Solver(mesh, grid, gas, W0, storage="f64") as s:
        dt = s.dt
    Wo, _, _, diag = O.run(mesh, grid, gas, W0, f0, 5, dt=dt)
    assert w_err(Wout, Wo) <= 1e-11
    np.testing.assert_allclose(res, diag[-1, :4], rtol=1e-9)


def test_nonphysical_state_is_reported(U):
    mesh, grid, gas, prim = cavity_case(n=8, nvx=10)
    W0 = I.prim_to_conservative(prim, 2, 0)
    with U.Solver(mesh, grid, gas, W0, storage="f64") as s:
        Wb, fb, _ = s.get_state()
        Wb[5, 0] = -1.0                     # negative density planted on the host
        s.set_state(Wb, fb, 0)
        s.step(1)
        with pytest.raises(U.UGKSError) as e:
            s.moments()
        assert e.value.status == 6


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32", 1e-5)])
@pytest.mark.parametrize("name", ["cavity_shakhov", "sphere_tet"])
def test_surface_quantities_match_oracle(U, name, storage, tol):
    """ugks_surface (reading R20: pressure, tangential stress and heat flux of
    every diffuse-wall face from the moments of its flux, and C_p, C_t, C_h)
    against the oracle's surface quantities after one step, element by element,
    relative to each quantity's largest magnitude."""
    mesh, grid, gas, prim = CASES[name]()
    W0 = I.prim_to_conservative(prim, mesh.dim, gas.K)
    far = [b for b in mesh.bc if b.type == I.BC_FARFIELD]
    ref = far[0] if far else mesh.bc[0]
    fs = [1.0] + [ref.u[d] if far else (0.14606 if d == 0 else 0.0) for d in range(mesh.dim)] + [1.0]
    with U.Solver(mesh, grid, gas, W0, storage=storage) as s:
        dt = s.dt
        s.step(1)
        faces, vals, coef = s.surface(fs)
        f2, v2, c2 = s.surface()
    _, _, _, _, F = O.run(mesh, grid, gas, W0, O.initial_f(mesh, grid, W0, gas.K), 1, dt=dt, face_flux=True)
    of, ov, oc = O.surface(mesh, F, dt, fs)
    assert len(faces) > 0 and np.array_equal(faces, of) and np.array_equal(f2, of) and c2 is None
    np.testing.assert_array_equal(vals, v2)
    for col in range(ov.shape[1]):
        scale = max(np.max(np.abs(ov[:, col])), np.max(np.abs(ov[:, 0])) * 1e-3)
        assert np.max(np.abs(vals[:, col] - ov[:, col])) <= tol * scale, (col, np.max(np.abs(vals[:, col] - ov[:, col])) / scale)
    for col in range(3):
        scale = np.max(np.abs(oc[:, col]))
        assert np.max(np.abs(coef[:, col] - oc[:, col])) <= tol * scale, col


def test_surface_is_refused_for_the_tiled_sweep(U):
    mesh, grid, gas, prim = cavity_case(n=8, nvx=10)
    with U.Solver(mesh, grid, gas, I.prim_to_conservative(prim, 2, 0), storage="f64", sweep="tiled") as s:
        s.step(1)
        with pytest.raises(U.UGKSError) as e:
            s.surface()
        assert e.value.status == 8


# Unit round-off of the scaled storage formats (11 and 8 significant bits).
STORAGE_EPS = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}


def _deviation_ratio(mesh, grid, gas, W, f):
    """max |f - g(W)| / max |f| per reduced distribution, g = the discrete
    Maxwellian of W (the reference the scaled storage encodes against)."""
    g = O.initial_f(mesh, grid, W, gas.K)
    return np.array([np.max(np.abs(f[r] - g[r])) / np.max(np.abs(f[r])) for r in range(f.shape[0])])


@pytest.mark.parametrize("sweep", ["scaled", "scaled_fused"])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_scaled_storage_one_step_matches_oracle(U, name, storage, sweep):
    """FP16 / BF16 deviations from a per-cell reference Maxwellian, FP32
    arithmetic.  f^0 is its own reference (zero deviations), so W after one step
    carries FP32 rounding only (<= 1e-5).  f^1 carries two storage roundings,
    each at most eps of the value's deviation from its reference (f~ against the
    Maxwellian of W^0, f^1 against that of W^1): per reduced distribution the
    error is within 1e-5 + 2 eps (D0 + D1) of max |f|, D0 and D1 the oracle's
    largest deviations from the two references.  Both organisations of the
    fluxes and first stage (split kernels, fused kernel)."""
    mesh, grid, gas, prim = CASES[name]()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 1, storage, sweep, key=name)
    W0 = I.prim_to_conservative(prim, mesh.dim, gas.K)
    assert w_err(Wg, Wo) <= 1e-5, w_err(Wg, Wo)
    dev = _deviation_ratio(mesh, grid, gas, W0, fo) + _deviation_ratio(mesh, grid, gas, Wo, fo)
    for r in range(fo.shape[0]):
        err = np.max(np.abs(fg[r] - fo[r])) / np.max(np.abs(fo[r]))
        assert err <= 1e-5 + 2 * STORAGE_EPS[storage] * dev[r], (r, err, dev[r])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("name", ["cavity_bgk", "periodic3d_bgk_K2", "strip1d_farfield_outflow"])
def test_scaled_storage_hundred_steps_matches_oracle(U, name, storage):
    """100 steps: each step adds to f at most eps times its deviation from the
    reference (at most 0.1 of max |f| in these cases), which moves W by at most
    that much per step (CFL < 1); accumulated linearly: W within 100 eps 0.1."""
    mesh, grid, gas, prim = CASES[name]()
    Wg, fg, res, Wo, fo, diag, dt, _ = run_pair(U, mesh, grid, gas, prim, 100, storage, "scaled", key="long_" + name)
    assert w_err(Wg, Wo) <= 100 * STORAGE_EPS[storage] * 0.1, w_err(Wg, Wo)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_scaled_storage_checkpoint_roundtrip(U, storage):
    """get_state / set_state re-encode f against the Maxwellian of the given W:
    a restart reproduces the continued run to the storage rounding of f."""
    mesh, grid, gas, prim = cavity_case(n=8, nvx=10)
    W0 = I.prim_to_conservative(prim, 2, 0)
    with U.Solver(mesh, grid, gas, W0, storage=storage) as s:
        s.step(3)
        W3, f3, k = s.get_state()
        s.step(4)
        W7 = s.moments()
    with U.Solver(mesh, grid, gas, W0, storage=storage) as s2:
        s2.set_state(W3, f3, 3)
        Wr, fr, _ = s2.get_state()
        np.testing.assert_array_equal(Wr, W3)
        assert np.max(np.abs(fr - f3)) <= STORAGE_EPS[storage] * np.max(np.abs(f3))
        s2.step(4)
        assert w_err(s2.moments(), W7) <= 4 * STORAGE_EPS[storage] * 0.1


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32", 1e-5)])
@pytest.mark.parametrize("name", ["cavity_shakhov", "periodic3d_bgk_K2", "cylinder_tri_K2"])
def test_moments13_and_chapman_enskog_start_match_oracle(U, name, storage, tol):
    """ugks_moments13 after two steps against the oracle's (reading R21), then
    ugks_init_moments13 of those fields against the oracle's Chapman-Enskog
    distribution and one further step."""
    mesh, grid, gas, prim = CASES[name]()
    W0 = I.prim_to_conservative(prim, mesh.dim, gas.K)
    with U.Solver(mesh, grid, gas, W0, storage=storage) as s:
        dt = s.dt
        s.step(2)
        m13 = s.moments13()
        s.init_moments13(m13)
        W1 = s.moments()
        fce = np.transpose(s.get_f(np.arange(mesh.n_cells)), (1, 0, 2))
        s.step(1)
        W2 = s.moments()
    Wo, fo, _, _ = O.run(mesh, grid, gas, W0, O.initial_f(mesh, grid, W0, gas.K), 2, dt=dt)
    mo = O.moments13(mesh.dim, gas.K, grid, Wo, fo)
    # rho, U, T relative to their largest magnitude; the stress P_ij - p delta_ij
    # and the heat flux are differences of O(p) moments, so their rounding is
    # relative to p (and p sqrt(T) for q)
    d, p = mesh.dim, 0.5 * mo[:, 0] * mo[:, mesh.dim + 1]
    for col in range(mo.shape[1]):
        if col <= d + 1:
            scale = np.max(np.abs(mo[:, col]))
        elif col < mo.shape[1] - d:
            scale = np.max(p)
        else:
            scale = np.max(p * np.sqrt(mo[:, d + 1]))
        assert np.max(np.abs(m13[:, col] - mo[:, col])) <= tol * scale, col
    fo_ce = O.chapman_enskog(mesh.dim, gas.K, grid, m13)
    assert rel_linf(fce, fo_ce, axis_fields=0) <= (1e-12 if storage == "f64" else 1e-6)
    Wc = np.zeros_like(W1)
    Wc[:, 0] = m13[:, 0]
    Wc[:, 1:1 + mesh.dim] = m13[:, :1][:, [0] * mesh.dim] * m13[:, 1:1 + mesh.dim]
    Wc[:, -1] = 0.5 * m13[:, 0] * np.sum(m13[:, 1:1 + mesh.dim] ** 2, axis=1) + (gas.K + 3) * m13[:, 0] * m13[:, mesh.dim + 1] / 4
    np.testing.assert_allclose(W1, Wc, rtol=1e-13)
    Wo2, _, _, _ = O.run(mesh, grid, gas, Wc, fo_ce, 1, dt=dt)
    assert w_err(W2, Wo2) <= tol, w_err(W2, Wo2)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32", 1e-5)])
@pytest.mark.parametrize("name", ["cavity_shakhov", "sphere_tet", "cylinder_tri_K2"])
def test_heat_flux_of_ugks_moments_matches_oracle(U, name, storage, tol):
    """ugks_moments' q (Eq. 13) of the state after two steps against the
    oracle's heat flux of the GPU's own f (h, b read back), per cell, relative
    to the largest |q| of the case."""
    mesh, grid, gas, prim = CASES[name]()
    W0 = I.prim_to_conservative(prim, mesh.dim, gas.K)
    with U.Solver(mesh, grid, gas, W0, storage=storage) as s:
        s.step(2)
        W, q = s.moments(with_q=True)
        f = s.get_f(np.arange(mesh.n_cells))               # [cell, r, k]
    qo = np.array([O.heat_flux(mesh.dim, gas.K, grid, f[i, 0], f[i, 1] if f.shape[1] == 2 else None, W[i])
                   for i in range(mesh.n_cells)])
    scale = np.abs(qo).max()
    assert scale > 0
    assert np.abs(q - qo).max() <= tol * scale
