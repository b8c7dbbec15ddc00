"""Pins of the oracle's planner network: the gradient against central finite
differences, closed forms of tiny networks, and Adam's first step."""

import numpy as np
import pytest

from oracle import mlp

DIMS = [5, 7, 6, 3]


def rand_problem(seed, n=11):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.param_count(DIMS)) * 0.5
    x = rng.standard_normal((n, DIMS[0]))
    t = rng.standard_normal((n, DIMS[-1]))
    return p, x, t


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_finite_differences(seed):
    p, x, t = rand_problem(seed)
    g = mlp.gradient(DIMS, p, x, t)
    h = 1e-6
    for k in range(0, len(p), 7):
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss(DIMS, p + e, x, t) - mlp.loss(DIMS, p - e, x, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-6 * abs(fd), (k, fd, g[k])


def test_linear_network_closed_form():
    # one layer: y = W x + b, loss = mean((y - t)^2); gradient 2/(n m) (y - t) x^T
    dims = [3, 2]
    rng = np.random.default_rng(4)
    W, b = rng.standard_normal((2, 3)), rng.standard_normal(2)
    p = np.concatenate([W.reshape(-1), b])
    x, t = rng.standard_normal((5, 3)), rng.standard_normal((5, 2))
    y = mlp.forward(dims, p, x)[-1]
    assert np.allclose(y, x @ W.T + b, atol=1e-15)
    r = 2 * (y - t) / y.size
    assert np.allclose(mlp.gradient(dims, p, x, t), np.concatenate([(r.T @ x).reshape(-1), r.sum(0)]))


def test_relu_blocks_negative_units():
    dims = [1, 2, 1]
    # hidden unit 0: relu(x), unit 1: relu(-x); output = unit0 - unit1 = x
    p = np.array([1.0, -1.0, 0.0, 0.0, 1.0, -1.0, 0.0])
    x = np.array([[2.0], [-3.0]])
    assert np.allclose(mlp.forward(dims, p, x)[-1], x)
    assert np.allclose(mlp.forward(dims, p, x)[0], [[2.0, 0.0], [0.0, 3.0]])


def test_adam_first_step_moves_every_parameter_by_lr():
    # bias-corrected first step: m/(1-b1) = g, v/(1-b2) = g^2, so dp = -lr sign(g)
    p, x, t = rand_problem(7)
    g = mlp.gradient(DIMS, p, x, t)
    p1, _, _, losses = mlp.adam_steps(DIMS, p, x, t, 1, 1e-3)
    nz = np.abs(g) > 1e-6
    assert np.allclose((p - p1)[nz], 1e-3 * np.sign(g[nz]), rtol=1e-4)
    assert losses[0] == pytest.approx(mlp.loss(DIMS, p, x, t))


def test_adam_fits_a_linear_map():
    dims = [2, 1]
    x = np.random.default_rng(1).standard_normal((64, 2))
    t = x @ np.array([[0.7], [-1.2]]) + 0.3
    p, _, _, losses = mlp.adam_steps(dims, np.zeros(3), x, t, 3000, 0.01)
    assert losses[-1] < 1e-6 and np.allclose(p, [0.7, -1.2, 0.3], atol=1e-3)
