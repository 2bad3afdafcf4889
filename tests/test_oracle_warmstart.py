"""Pins of the oracle's learned-warm-start pieces: kNN by an independent distance sort, rotation and
translation invariance of the features, coefficients that reproduce a retained-space density exactly,
MLP gradients against central finite differences, and Adam reducing the loss on a fixed batch."""
import numpy as np

import oracle
from oracle import warmstart as ws
import suspensions


def test_neighbours_match_a_distance_sort():
    s = suspensions.random_ellipsoids(40, 4, 8, 0.1, 0.2, seed=3)
    nb = ws.neighbours(s.centres)
    d = np.linalg.norm(s.centres[:, None] - s.centres[None], axis=2)
    for i in (0, 7, 39):
        order = [j for j in np.lexsort((np.arange(40), d[i])) if j != i][:16]
        assert nb[i] == order


def test_features_invariant_under_rigid_motion():
    s = suspensions.random_ellipsoids(20, 4, 8, 0.1, 0.2, seed=4)
    X0 = ws.features(s.semi_axes, s.centres, s.quats, s.F, s.T)
    qg = np.array([0.8, 0.2, -0.5, 0.26])
    qg /= np.linalg.norm(qg)
    Q = oracle.quat_to_rot(qg)
    from oracle.timestep import quat_mul
    rot_q = quat_mul(np.tile(qg, (20, 1)), s.quats)
    X1 = ws.features(s.semi_axes, s.centres @ Q.T + 3.0, rot_q, s.F @ Q.T, s.T @ Q.T)
    assert np.abs(X1 - X0).max() < 1e-12
    assert np.all(X0[:, 121:] == 0) and np.allclose(X0[:, 6:9], s.semi_axes)


def test_coefficients_round_trip_on_retained_space():
    s = suspensions.random_ellipsoids(3, 6, 14, 0.05, 0.3, seed=5)
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    nb = (6 + 1) ** 2
    coef = np.random.default_rng(1).normal(size=(3, 3 * nb))
    mu = ws.synthesize(ref, coef)
    assert np.abs(ws.target_coefficients(ref, mu) - coef).max() < 1e-12


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = ws.init_params(12, seed=3)
    X = rng.normal(size=(5, 128))
    Y = rng.normal(size=(5, 12))
    L, g = ws.loss_and_grads(params, X, Y)
    for k, idx in [("W1", (3, 7)), ("b1", (11,)), ("W2", (100, 5)), ("b2", (0,)), ("W3", (17, 4)), ("b3", (9,))]:
        h = 1e-6
        p = {a: b.copy() for a, b in params.items()}
        p[k][idx] += h
        Lp, _ = ws.loss_and_grads(p, X, Y)
        p[k][idx] -= 2 * h
        Lm, _ = ws.loss_and_grads(p, X, Y)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[k][idx]) < 1e-6 * max(1.0, abs(fd)), k


def test_gelu_matches_its_definition_and_derivative():
    x = np.linspace(-5, 5, 101)
    assert np.allclose(ws.gelu(x), 0.5 * x * (1 + np.tanh(np.sqrt(2 / np.pi) * (x + 0.044715 * x ** 3))))
    h = 1e-6
    assert np.allclose(ws.gelu_grad(x), (ws.gelu(x + h) - ws.gelu(x - h)) / (2 * h), atol=1e-8)


def test_adam_fits_a_fixed_batch():
    rng = np.random.default_rng(4)
    params = ws.init_params(6, seed=5)
    X = rng.normal(size=(64, 128))
    Y = np.tanh(X[:, :6])
    state = {}
    L0, _ = ws.loss_and_grads(params, X, Y)
    for _ in range(200):
        L, g = ws.loss_and_grads(params, X, Y)
        ws.adam_step(params, g, state, lr=1e-3)
    assert L < 0.05 * L0
