"""Warm-start network (ugks_mlp_*) against the FP64 reference network.

The GPU network keeps BF16 weights and activations with FP32 accumulation.
The reference is given the same BF16-rounded weights and inputs, so the
remaining differences come from rounding the hidden activations and the
back-propagated gradients to BF16 (relative 2^-9 per rounding) and from FP32
summation order.  Over L layers these add up to about L * 2^-9 relative; the
bounds below are four times that, relative to the largest magnitude of the
compared array."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as MO
from paper_2606_15720_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BF16_EPS = 2.0 ** -9


def bf16_round(x):
    """Round to the nearest BF16 (ties to even) through the FP32 bit pattern."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def make_net(sizes, seed=0):
    from paper_2606_15720_gb300 import ugks as U
    net = U.WarmStartNet(sizes[0], sizes[-1], width=sizes[1], hidden_layers=len(sizes) - 2, seed=seed)
    params = MO.init_params(sizes, seed=seed)
    net.set_params(MO.flatten(params).astype(np.float32))
    return net, params


def rounded(params):
    """The parameters the GPU computes with: BF16 weights, FP32 biases."""
    return [(bf16_round(W), b.astype(np.float32).astype(np.float64)) for W, b in params]


SHAPES = {"small_ragged": [6, 40, 40, 40, 9], "warm_start_6x256": [6] + [256] * 6 + [9]}


def test_param_roundtrip_is_exact():
    net, params = make_net(SHAPES["small_ragged"], seed=3)
    ref = MO.flatten(params).astype(np.float32)
    assert net.param_count() == ref.size
    np.testing.assert_array_equal(net.get_params(), ref)


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("n", [300, 4096])
def test_forward_matches_reference(shape, n):
    sizes = SHAPES[shape]
    net, params = make_net(sizes, seed=1)
    rng = np.random.default_rng(2)
    X = rng.uniform(-2.0, 2.0, (n, sizes[0])).astype(np.float32)
    y = net.predict(X)
    y_ref, _ = MO.forward(rounded(params), bf16_round(X))
    L = len(sizes) - 1
    tol = 4 * L * BF16_EPS * np.abs(y_ref).max()
    assert np.abs(y - y_ref).max() <= tol


@pytest.mark.parametrize("shape", list(SHAPES))
def test_gradients_match_reference(shape):
    sizes = SHAPES[shape]
    net, params = make_net(sizes, seed=5)
    rng = np.random.default_rng(6)
    n = 700                                         # 11 tiles of 64 samples, ragged
    X = rng.uniform(-2.0, 2.0, (n, sizes[0])).astype(np.float32)
    T = rng.normal(size=(n, sizes[-1])).astype(np.float32)
    g, loss = net.gradients(X, T)
    p_ref = rounded(params)
    g_ref = MO.flatten(MO.gradients(p_ref, bf16_round(X), T.astype(np.float64)))
    loss_ref = MO.loss(p_ref, bf16_round(X), T.astype(np.float64))
    L = len(sizes) - 1
    assert abs(loss - loss_ref) <= 4 * L * BF16_EPS * loss_ref
    o = 0
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        for size in (fan_in * fan_out, fan_out):
            a, b = g[o:o + size], g_ref[o:o + size]
            o += size
            scale = np.abs(b).max()
            assert np.abs(a - b).max() <= 4 * L * BF16_EPS * scale
            assert np.linalg.norm(a - b) <= 4 * L * BF16_EPS * np.linalg.norm(b)


def test_adam_first_step_matches_reference():
    """Adam's first bias-corrected step is lr * g / (|g| + eps): lr against
    the sign of every gradient component that is not tiny."""
    sizes = SHAPES["small_ragged"]
    net, params = make_net(sizes, seed=7)
    rng = np.random.default_rng(8)
    n = 500
    X = rng.uniform(-2.0, 2.0, (n, sizes[0])).astype(np.float32)
    T = rng.normal(size=(n, sizes[-1])).astype(np.float32)
    lr = 1e-3
    p0 = net.get_params().astype(np.float64)
    net.train(X, T, epochs=1, batch=n, lr=lr, seed=0)    # one Adam step on the whole set
    p1 = net.get_params().astype(np.float64)
    p_ref = rounded(params)
    g_ref = MO.flatten(MO.gradients(p_ref, bf16_round(X), T.astype(np.float64)))
    new_ref, _ = MO.adam_step(MO.unflatten(p0, sizes), MO.unflatten(g_ref, sizes), None, lr)
    new_ref = MO.flatten(new_ref)
    big = np.abs(g_ref) > 0.05 * np.abs(g_ref).max()
    assert big.sum() > 100
    np.testing.assert_allclose(p1[big], new_ref[big], rtol=0, atol=1e-3 * lr + 1e-6)
    assert np.all(np.abs(p1 - p0) <= lr * (1 + 1e-3) + 1e-6)


def test_training_fits_a_teacher_network():
    """Adam on the GPU drives the loss on a target drawn from a smaller
    network far below its starting value; the padding of the layer widths
    stays zero (re-setting the read-back parameters changes no prediction)."""
    rng = np.random.default_rng(11)
    teacher = MO.init_params([6, 16, 9], seed=12)
    X = rng.uniform(-1.5, 1.5, (6000, 6))
    Y, _ = MO.forward(teacher, X)
    sizes = [6, 48, 48, 48, 9]
    net, _ = make_net(sizes, seed=13)
    _, loss0 = net.gradients(X[:4096], Y[:4096])
    loss = net.train(X, Y, epochs=60, batch=256, lr=2e-3, seed=1)
    assert np.isfinite(loss) and loss < 0.02 * loss0
    before = net.predict(X[:1000])
    net.set_params(net.get_params())
    np.testing.assert_array_equal(net.predict(X[:1000]), before)


def test_features_and_wall_distance():
    from paper_2606_15720_gb300 import ugks as U
    mesh = I.cylinder_tri_mesh(600, seed=3, mach=2.0)
    net = U.WarmStartNet(6, 9, width=16, hidden_layers=1)
    F = net.features(mesh, 2.0, 0.1)
    assert F.shape == (mesh.n_cells, 6)
    np.testing.assert_array_equal(F[:, 0], np.float32(2.0))
    np.testing.assert_array_equal(F[:, 1], np.float32(-1.0))
    np.testing.assert_array_equal(F[:, 2:4], mesh.cell_centroid.astype(np.float32))
    np.testing.assert_array_equal(F[:, 4], 0.0)
    walls = [b for b, bc in enumerate(mesh.bc) if bc.type == I.BC_WALL]
    wf = np.isin(-mesh.face_neighbor - 1, walls) & (mesh.face_neighbor < 0)
    d = np.sqrt(((mesh.cell_centroid[:, None, :] - mesh.face_centroid[None, wf, :]) ** 2).sum(-1)).min(1)
    np.testing.assert_allclose(F[:, 5], d.astype(np.float32), rtol=1e-6, atol=0)


def _cavity_solver(U):
    from test_gpu_parity import cavity_case
    mesh, grid, gas, prim = cavity_case(n=10, nvx=28)
    return mesh, U.Solver(mesh, grid, gas, I.prim_to_conservative(prim, 2, gas.K), storage="f32")


def test_warm_start_sets_the_predicted_fields_and_falls_back_to_freestream():
    """A network with zero weights predicts its last bias everywhere; the warm
    start sets the Chapman-Enskog state of those fields (its moments give them
    back up to the grid's quadrature error), scales stress and heat flux
    above the bound down, and replaces non-physical predictions by the
    freestream."""
    from paper_2606_15720_gb300 import ugks as U
    mesh, s = _cavity_solver(U)
    sizes = [6, 32, 32, 9]
    net = U.WarmStartNet(6, 9, width=32, hidden_layers=2)
    fields = np.array([1.2, 0.3, -0.1, 1.1, 0.02, -0.01, -0.015, 0.01, -0.005])
    p = np.zeros(net.param_count(), dtype=np.float32)
    p[-9:] = fields
    net.set_params(p)
    fs = np.array([1.0, 0.0, 0.0, 1.0])
    nf = net.warm_start(s, mesh, 0.16, 0.075, fs)
    assert nf == 0
    m13 = s.moments13()
    np.testing.assert_allclose(m13[:, :4], np.broadcast_to(fields[:4], (mesh.n_cells, 4)), rtol=0, atol=2e-4)
    np.testing.assert_allclose(m13[:, 4:], np.broadcast_to(fields[4:], (mesh.n_cells, 5)), rtol=0, atol=2e-3)
    # stress above p/2 (p = rho T / 2 = 0.66): stress and heat flux scaled by 0.33 / 1.32
    big = fields.copy()
    big[4] = 1.32
    p[-9:] = big
    net.set_params(p)
    assert net.warm_start(s, mesh, 0.16, 0.075, fs) == 0
    m13 = s.moments13()
    alpha = 0.5 * 0.66 / 1.32
    np.testing.assert_allclose(m13[:, :4], np.broadcast_to(big[:4], (mesh.n_cells, 4)), rtol=0, atol=2e-4)
    np.testing.assert_allclose(m13[:, 4:], np.broadcast_to(alpha * big[4:], (mesh.n_cells, 5)), rtol=0, atol=2e-3)
    p[-9:] = fields
    p[-9] = -1.0                                   # rho < 0: every cell falls back
    net.set_params(p)
    nf = net.warm_start(s, mesh, 0.16, 0.075, fs)
    assert nf == mesh.n_cells
    m13 = s.moments13()
    np.testing.assert_allclose(m13[:, :4], np.broadcast_to(fs, (mesh.n_cells, 4)), rtol=0, atol=2e-4)
    np.testing.assert_allclose(m13[:, 4:], 0.0, rtol=0, atol=2e-3)
    del sizes


def test_trained_warm_start_reaches_steady_state_sooner():
    """The gain of the learned warm start.  Six cylinder cases (Ma 1.5-3,
    Kn 0.1-0.4, about 700 triangles, 24^2 velocities) converged by the solver
    train the 6x256 network; a held-out case on a new mesh (Ma 1.9, Kn 0.2)
    then reaches the density residual 1e-6 in fewer steps and less time from
    the warm start than from the freestream, and reaches the accuracy of the
    freestream solve (every field at least as close to the solve continued to
    1e-8) sooner too."""
    from paper_2606_15720_gb300 import warmstart as WS
    train = [(ma, kn) for ma in (1.5, 2.25, 3.0) for kn in (0.1, 0.4)]
    res = WS.experiment(train, [(1.9, 0.2)], cells=700, nvx=24, schedule=((150, 1e-3), (100, 3e-4)), batch=256,
                        ref_tol=1e-8, max_steps=80_000)
    assert all(n is not None for n in res["train_converge"]["steps"])
    assert res["training"]["loss"][-1] < 0.01
    c = res["cases"][0]
    assert c["warm"]["fallback_cells"] == 0
    assert c["step_ratio"] > 1.2 and c["time_ratio"] > 1.2
    assert c["equal_accuracy_step_ratio"] > 1.2
    warm0, free0 = c["initial_error_vs_reference"]["warm"], c["initial_error_vs_reference"]["freestream"]
    assert all(a < 0.5 * b for a, b in zip(warm0, free0))
