"""Oracle pins for the stopping/lambda network (FD gradients, GELU, Adam)."""
import math

import numpy as np

from oracle import mlp


def test_param_count():
    assert mlp.N_PARAMS == 20 * 128 + 128 + 128 * 128 + 128 + 128 * 2 + 2 == 19458


def test_gelu_against_math_erf_and_limits():
    for z in (-5.0, -1.3, -0.2, 0.0, 0.7, 3.1):
        ref = 0.5 * z * (1 + math.erf(z / math.sqrt(2)))
        assert abs(mlp.gelu(np.array([z]))[0] - ref) < 1e-15
    z = np.linspace(-4, 4, 81)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8
    assert mlp.gelu(np.array([40.0]))[0] == 40.0 and mlp.gelu(np.array([-40.0]))[0] == 0.0


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(3)
    X = rng.normal(size=(7, 20))
    T = rng.normal(size=(7, 2))
    L, g = mlp.loss_and_grad(theta, X, T)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 2559, 2560 + 127, 19457, 19456]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, T)[0] - mlp.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, i


def test_adam_first_step_is_sign_step():
    # with m = v = 0, the bias-corrected first step is lr * g / (|g| + eps) ~ lr * sign(g)
    theta = np.zeros(5)
    g = np.array([2.0, -0.5, 1e-3, -3.0, 0.0])
    th, m, v = mlp.adam_step(theta, np.zeros(5), np.zeros(5), g, 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_reduces_loss():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(64, 20))
    T = np.stack([np.tanh(X[:, 0]), X[:, 1] * 0.5], axis=1)
    theta = mlp.init_params(1)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = mlp.loss_and_grad(theta, X, T)[0]
    for t in range(1, 201):
        L, g = mlp.loss_and_grad(theta, X, T)
        theta, m, v = mlp.adam_step(theta, m, v, g, t, lr=3e-3)
    assert mlp.loss_and_grad(theta, X, T)[0] < 0.1 * L0
