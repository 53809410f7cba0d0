"""Pins of the FP64 surrogate-network oracle: the analytic gradient against central
finite differences, the first Adam step's closed form, bfloat16 rounding against
torch's conversion, and a loss that falls on a fixed seed."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _problem(seed=0, B=40):
    rng = np.random.default_rng(seed)
    n = sum(int(np.prod(s)) for s in mlp.sizes())
    theta = rng.normal(0, 0.3, n)
    X = rng.normal(2.0, 3.0, (B, 6))
    Y = rng.normal(0, 1.0, (B, 3))
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    return theta, X, Y, mean, std


def test_gradient_matches_central_differences():
    theta, X, Y, mean, std = _problem()
    loss, g = mlp.loss_and_grad(theta, X, Y, mean, std)
    rng = np.random.default_rng(5)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tp[i] += h
        tm = theta.copy()
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, Y, mean, std)[0] - mlp.loss_and_grad(tm, X, Y, mean, std)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_zero_weights_output_bias():
    theta, X, Y, mean, std = _problem()
    W1, b1, W2, b2, W3, b3 = mlp.unflatten(theta)
    t2 = mlp.flatten([W1, b1, W2, b2, np.zeros_like(W3), np.array([0.5, -1.0, 2.0])])
    y, _ = mlp.forward(t2, X, mean, std)
    np.testing.assert_array_equal(y, np.broadcast_to([0.5, -1.0, 2.0], y.shape))


def test_first_adam_step_is_signed_lr():
    theta, X, Y, mean, std = _problem()
    _, g = mlp.loss_and_grad(theta, X, Y, mean, std)
    new, m, v = mlp.adam_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3)
    big = np.abs(g) > 1e-3
    np.testing.assert_allclose((theta - new)[big], 1e-3 * np.sign(g[big]), rtol=1e-4)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.normal(0, 1, 1000), [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5e-3, 0.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.round_bf16(a), ref)


def test_adam_reduces_the_loss():
    theta, X, Y, mean, std = _problem(B=200)
    # a learnable target: a smooth function of the inputs
    Y = np.stack([np.sin(X[:, 0] / 3), np.tanh(X[:, 1] - X[:, 2]) * 0.5, 0.1 * X[:, 3]], axis=1)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0 = mlp.loss_and_grad(theta, X, Y, mean, std)[0]
    for t in range(1, 301):
        loss, g = mlp.loss_and_grad(theta, X, Y, mean, std)
        theta, m, v = mlp.adam_step(theta, g, m, v, t, lr=3e-3)
    assert loss < 0.2 * l0
