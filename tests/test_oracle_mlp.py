"""Pins of the FP64 network oracle: back-propagation against central finite
differences of the loss, and Adam's defining properties."""
import numpy as np
import pytest

from oracle import mlp


def test_param_count():
    assert mlp.N_PARAMS == 4675


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(3) + 0.05 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.uniform(-1, 1, (17, 4))
    T = rng.standard_normal((17, 3))
    _, g = mlp.gradient(theta, X, T)
    idx = rng.choice(mlp.N_PARAMS, 120, replace=False)
    idx = np.concatenate([idx, [0, 255, 256, 319, 320, 4415, 4416, 4479, 4480, 4671, 4672, 4674]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_zero_gradient_at_a_perfect_fit():
    theta = mlp.init_params(5)
    X = np.random.default_rng(2).uniform(-1, 1, (9, 4))
    T, _ = mlp.forward(theta, X)
    loss, g = mlp.gradient(theta, X, T)
    assert loss == 0.0 and np.max(np.abs(g)) == 0.0


def test_first_adam_step_moves_each_parameter_by_lr_times_sign():
    """With zero moments, Adam's bias-corrected first step is
    -lr * g / (|g| + eps), i.e. -lr sign(g) wherever |g| >> eps."""
    theta = mlp.init_params(7)
    rng = np.random.default_rng(3)
    X, T = rng.uniform(-1, 1, (8, 4)), rng.standard_normal((8, 3))
    _, g = mlp.gradient(theta, X, T)
    new, _ = mlp.adam_train(theta, X, T, np.arange(8)[None, :], batch=8, lr=1e-3)
    big = np.abs(g) > 1e-5
    assert np.allclose((new - theta)[big], -1e-3 * np.sign(g[big]), rtol=1e-3)


def test_adam_fits_a_smooth_map():
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (256, 4))
    T = np.stack([np.sin(X[:, 0]) + X[:, 1] ** 2, X[:, 2] * X[:, 3], np.cos(X.sum(1))], 1)
    theta = mlp.init_params(0)
    order = np.stack([rng.permutation(256) for _ in range(200)])
    l0 = mlp.loss(theta, X, T)
    theta, _ = mlp.adam_train(theta, X, T, order, batch=64, lr=3e-3)
    assert mlp.loss(theta, X, T) < 0.05 * l0
