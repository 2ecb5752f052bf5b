"""Batches of cases stepped through one CUDA graph (ugks_batch_*).

Heterogeneous cases (2-D quads, 2-D triangles with K = 2, 3-D periodic box)
in one batch: a graph launch advances every case by two steps on forked
streams.  The per-case arithmetic is the ordinary step's, so batch results
equal the cases stepped one by one (W bitwise at the same block size; the
residual up to the summation order of its atomics) and
match the oracle; the block-size autotuner picks one of the allowed sizes and
caches it per case shape."""
import numpy as np
import pytest

import oracle as O
from paper_2606_15720_gb300 import inputs as I

from test_gpu_parity import cavity_case, cylinder_case, periodic3d_case, w_err

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    for mesh, grid, gas, prim in (cavity_case(n=12, nvx=14), cylinder_case(cells=900, nvx=11), periodic3d_case()):
        out.append((mesh, grid, gas, I.prim_to_conservative(prim, mesh.dim, gas.K)))
    return out


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("nsteps", [4, 3])
def test_batch_graph_steps_equal_single_case_steps(nsteps, storage):
    from paper_2606_15720_gb300 import ugks as U
    cases = _cases()
    with U.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases],
                 storage=storage, block_velocities=64) as b:
        b.step(nsteps)
        Wb = [s.moments() for s in b.cases]
        rb = [s.residual() for s in b.cases]
    for (mesh, grid, gas, W0), W, r in zip(cases, Wb, rb):
        with U.Solver(mesh, grid, gas, W0, storage=storage, sweep="blocked", block_velocities=64) as s:
            s.step(nsteps)
            np.testing.assert_array_equal(W, s.moments())
            # the residual's cross-CTA sum uses atomics: equal up to summation order
            np.testing.assert_allclose(r, s.residual(), rtol=1e-13, atol=0)


def test_batch_fp64_matches_oracle():
    from paper_2606_15720_gb300 import ugks as U
    cases = _cases()
    with U.Batch([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases],
                 storage="f64") as b:
        b.step(4)
        res = [(s.moments(), s.dt) for s in b.cases]
    for (mesh, grid, gas, W0), (W, dt) in zip(cases, res):
        Wo, _, _, _ = O.run(mesh, grid, gas, W0, O.initial_f(mesh, grid, W0, gas.K), 4, dt=dt)
        assert w_err(W, Wo) <= 1e-11, w_err(W, Wo)


def test_autotuner_picks_an_allowed_block_size_and_caches_it():
    from paper_2606_15720_gb300 import ugks as U
    cases = _cases()
    args = ([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases])
    with U.Batch(*args, storage="f32") as b:
        b.autotune()
        picks = [b.tuning(i) for i in range(len(cases))]
        for bv, ms in picks:
            assert bv in (32, 64, 128, 256)
            assert ms[0] > 0.0 and ms[{32: 0, 64: 1, 128: 2, 256: 3}[bv]] == pytest.approx(min(m for m in ms if m > 0))
        for s in b.cases:
            assert np.all(np.isfinite(s.moments()))
    # the same case shapes again: the cached sizes are reused, no tuning steps run
    with U.Batch(*args, storage="f32") as b2:
        b2.autotune()
        for i, (bv, _) in enumerate(picks):
            bv2, ms2 = b2.tuning(i)
            assert bv2 == bv and np.all(ms2 == 0.0)
            np.testing.assert_array_equal(b2.cases[i].moments(), cases[i][3])


def test_autotuner_shapes_are_allowed_and_keep_the_cases_physical():
    """The shape search (block size, split or fused fluxes and first stage,
    second-stage chunks) returns an allowed shape per case, and stepping with
    it matches a case stepped with the same block size and organisation to
    FP32 rounding (the chunk count changes only the heat flux's summation
    order)."""
    from paper_2606_15720_gb300 import ugks as U
    cases = _cases()
    args = ([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases])
    with U.Batch(*args, storage="f32") as b:
        b.autotune()
        shapes = [b.shape(i) for i in range(len(cases))]
        states = [s.get_state() for s in b.cases]
        b.step(2)
        W_after = [s.moments() for s in b.cases]
    for (mesh, grid, gas, W0), sh, (Ws, fs, k), Wa in zip(cases, shapes, states, W_after):
        assert sh["block_velocities"] in (32, 64, 128, 256)
        assert sh["stage2_chunks"] >= 1
        # tuned here (at least the block sizes, the organisation and one chunk count), or reused from the
        # process cache when an earlier batch tuned the same case shape
        assert (sh["trials"] >= 3 and sh["ms_per_step"] > 0.0) or (sh["trials"] == 0 and sh["ms_per_step"] == 0.0)
        with U.Solver(mesh, grid, gas, W0, storage="f32", block_velocities=sh["block_velocities"],
                      sweep="blocked_fused" if sh["fused"] else "blocked") as s:
            s.set_state(Ws, fs, k)
            s.step(2)
            assert w_err(Wa, s.moments()) <= 1e-6, w_err(Wa, s.moments())


def test_autotuned_batch_of_cylinders_stays_physical_after_memory_reuse():
    """Eight cases of the cylinder batch workload (5k-40k triangles, padded
    velocity grids): a first batch is created, stepped and freed, so that a
    second one reuses its device memory; the second is autotuned and stepped;
    every case stays physical.  Its shapes include the fused flux +
    first-stage kernel, which reads every lane of the per-face buffer (lanes
    with u.n = 0, padding included, must be written by the reconstruction
    each block), and second-stage chunk counts of 1-4, where one CTA streams
    many velocity rows through its ring of shared-memory stages (a stage must
    not be refilled before the rows read from it have been used)."""
    import bench
    from paper_2606_15720_gb300 import ugks as U
    cases = bench.batch_cases(n=8)
    args = ([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases])
    with U.Batch(*args, storage="f32") as b:
        b.step(4)
    with U.Batch(*args, storage="f32") as b:
        b.autotune()
        b.step(6)
        for s in b.cases:
            s.residual()                                   # raises on a non-physical state
            assert np.all(np.isfinite(s.moments()))
