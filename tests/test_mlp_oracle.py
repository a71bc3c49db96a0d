"""Pins of the FP64 fold-in MLP oracle: a hand-computed forward pass, central
finite differences of the loss for every parameter, and the Adam step against
its first-step closed form (|step| = lr when the bias corrections cancel)."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_forward_hand_computed():
    # 2 inputs -> 2 hidden -> 2 hidden -> 1 output, one sample
    W1 = np.array([[1.0, -1.0], [0.5, 2.0]])
    b1 = np.array([0.0, 0.5])
    W2 = np.array([[1.0, 0.0], [-1.0, 1.0]])
    b2 = np.array([0.25, -0.5])
    W3 = np.array([[2.0], [1.0]])
    b3 = np.array([-1.0])
    x = np.array([[1.0, 2.0]])
    # z1 = [1*1 + 2*0.5, 1*-1 + 2*2] + [0, .5] = [2, 3.5]; h1 = [2, 3.5]
    # z2 = [2*1 + 3.5*-1, 2*0 + 3.5*1] + [.25, -.5] = [-1.25, 3.0]; h2 = [0, 3]
    # z3 = 0*2 + 3*1 - 1 = 2; out = log(1 + e^2)
    out, _ = mlp.forward([W1, b1, W2, b2, W3, b3], x)
    assert out[0, 0] == pytest.approx(math.log1p(math.exp(2.0)), rel=1e-15)


def test_gradient_by_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init_params((6, 5, 4, 3), seed=1)
    params = [p + rng.uniform(-0.1, 0.1, p.shape) for p in params]  # nonzero biases
    x = rng.uniform(0.0, 2.0, (3, 6))
    t = rng.gamma(0.5, 1.0, (3, 3))
    out, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, t)
    for k, p in enumerate(params):
        flat = p.reshape(-1)
        g = grads[k].reshape(-1)
        for e in range(flat.size):
            h = 1e-6
            old = flat[e]
            flat[e] = old + h
            lp = mlp.loss(mlp.forward(params, x)[0], t)
            flat[e] = old - h
            lm = mlp.loss(mlp.forward(params, x)[0], t)
            flat[e] = old
            fd = (lp - lm) / (2 * h)
            assert g[e] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, e)


def test_adam_first_step():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    st = mlp.adam_state(p)
    mlp.adam_step(p, g, st, lr=0.1, t=1)
    # first step: m_hat = g, v_hat = g^2, so the step is lr * g / (|g| + eps) ~ lr * sign(g)
    np.testing.assert_allclose(p[0], [0.9, -1.9, 2.9], rtol=0, atol=1e-5)


def test_training_reduces_loss():
    rng = np.random.default_rng(2)
    params = mlp.init_params((20, 16, 16, 4), seed=3)
    x = rng.uniform(0, 1, (64, 20))
    t = np.log1p(np.exp(x[:, :4] @ rng.uniform(0, 1, (4, 4))))
    st = mlp.adam_state(params)
    l0 = mlp.loss(mlp.forward(params, x)[0], t)
    for step in range(1, 201):
        out, cache = mlp.forward(params, x)
        mlp.adam_step(params, mlp.backward(params, cache, t), st, 1e-2, step)
    assert mlp.loss(mlp.forward(params, x)[0], t) < 0.2 * l0
