"""Pins of the MLP oracle: back-propagation against central finite differences of its own
forward pass (a check independent of the backward code), special cases with closed forms,
the feature layout, and an Adam step against its defining recursion on a scalar."""
import math

import numpy as np

from oracle import mlp
from oracle import modes as md


def test_gradient_matches_finite_differences():
    H = 12
    g = np.random.default_rng(1)
    theta = mlp.init(H, 3) + 0.01 * g.standard_normal(mlp.n_params(H))
    x = g.standard_normal((7, mlp.D_IN))
    t = g.standard_normal(7)
    _, grad = mlp.loss_and_grad(theta, H, x, t)
    for i in g.choice(len(theta), 60, replace=False):
        e = np.zeros_like(theta)
        e[i] = 1e-6
        fd = (mlp.loss_and_grad(theta + e, H, x, t)[0] - mlp.loss_and_grad(theta - e, H, x, t)[0]) / 2e-6
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_closed_forms():
    H = 5
    x = np.random.default_rng(2).standard_normal((4, mlp.D_IN))
    # all weights zero: y = b3 for every input, and only b3 gets a gradient
    theta = np.zeros(mlp.n_params(H))
    theta[-1] = 0.7
    y, _ = mlp.forward(theta, H, x)
    assert np.allclose(y, 0.7)
    t = np.array([1.0, 0.0, -1.0, 2.0])
    loss, grad = mlp.loss_and_grad(theta, H, x, t)
    assert math.isclose(loss, np.mean((0.7 - t) ** 2))
    assert np.allclose(grad[:-1], 0) and math.isclose(grad[-1], 2 * np.mean(0.7 - t))
    # identity-like network on positive inputs: W1 = [I 0], W2 = I, w3 = 1 -> y = sum of the first H inputs
    W1 = np.zeros((H, mlp.D_IN))
    W1[:, :H] = np.eye(H)
    theta = np.concatenate([W1.ravel(), np.zeros(H), np.eye(H).ravel(), np.zeros(H), np.ones(H), np.zeros(1)])
    xp = np.abs(x)
    assert np.allclose(mlp.forward(theta, H, xp)[0], xp[:, :H].sum(1))


def test_features_layout():
    L = 12
    nn, nr = md.momenta_n(L, md.NS), md.momenta_n(L, md.R)
    x = mlp.features(L, [(0, 5)], [(1, 11)], nn, nr)[0]
    assert x[0] == nn[0] / L and x[1] == nn[5] / L and np.all(x[2:mlp.Q] == 0)
    assert x[mlp.Q] == nr[1] / L and x[mlp.Q + 1] == 1.0          # k = pi
    assert x[2 * mlp.Q] == 2 / mlp.Q and x[2 * mlp.Q + 2] == 2.0 and x[2 * mlp.Q + 3] == 1.0
    y = mlp.target(48, np.array([1e-3, 0.0]), [2, 0], [2, 0])
    assert math.isclose(y[0], -3 + 2 * math.log10(2)) and y[1] == -30.0


def test_adam_scalar_recursion():
    theta, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    g = np.array([0.5])
    th1, m1, v1 = mlp.adam_step(theta, g, m, v, 1, lr=0.1)
    # first step with bias correction moves by lr * g / (|g| + eps) ~ lr * sign(g)
    assert math.isclose(th1[0], 1.0 - 0.1 * 0.5 / (0.5 + 1e-8))
    assert math.isclose(m1[0], 0.05) and math.isclose(v1[0], 0.001 * 0.25)
