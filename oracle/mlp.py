"""FP64 oracle of the fold-in encoder MLP (test infrastructure only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The encoder maps one slice Y[i, :, :] of a CP model 'ir,jr,kr->ijk' to its
nonnegative loading row A[i, :] (the factor row that the multiplicative update
of mode 0 with B, C fixed would produce):

    x   = log1p(slice), flattened (J*K inputs)
    h1  = relu(x  W1 + b1)
    h2  = relu(h1 W2 + b2)
    out = softplus(h2 W3 + b3)                 (nonnegative loadings)
    L   = mean over batch and outputs of (log1p(out) - log1p(target))^2

Weights are stored [fan_in x fan_out] (row-major).  Training uses Adam
(Kingma & Ba): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

This module writes the forward pass, its gradient by the chain rule, and the
optimizer step out plainly with numpy matrix products (a library primitive).
"""
from __future__ import annotations

import numpy as np


def softplus(z):
    # log(1 + e^z), written to stay finite for large |z|
    return np.where(z > 30.0, z, np.log1p(np.exp(np.minimum(z, 30.0))))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def init_params(sizes, seed=0):
    """He-uniform weights, zero biases; sizes = (n_in, h1, h2, n_out)."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / a)
        params.append(rng.uniform(-lim, lim, size=(a, b)))
        params.append(np.zeros(b))
    return params


def forward(params, x):
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3 + b3
    out = softplus(z3)
    return out, (x, z1, h1, z2, h2, z3, out)


def loss(out, target):
    d = np.log1p(out) - np.log1p(target)
    return float(np.mean(d * d))


def backward(params, cache, target):
    """Gradients of `loss` with respect to (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    x, z1, h1, z2, h2, z3, out = cache
    n = out.size
    d = np.log1p(out) - np.log1p(target)
    g_out = 2.0 * d / (1.0 + out) / n          # dL/dout
    g_z3 = g_out * sigmoid(z3)                 # softplus' = sigmoid
    gW3 = h2.T @ g_z3
    gb3 = g_z3.sum(axis=0)
    g_h2 = g_z3 @ W3.T
    g_z2 = g_h2 * (z2 > 0.0)
    gW2 = h1.T @ g_z2
    gb2 = g_z2.sum(axis=0)
    g_h1 = g_z2 @ W2.T
    g_z1 = g_h1 * (z1 > 0.0)
    gW1 = x.T @ g_z1
    gb1 = g_z1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state = list of (m, v) per parameter; t >= 1."""
    for k, (p, g) in enumerate(zip(params, grads)):
        m, v = state[k]
        m *= b1
        m += (1.0 - b1) * g
        v *= b2
        v += (1.0 - b2) * g * g
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)


def adam_state(params):
    return [(np.zeros_like(p), np.zeros_like(p)) for p in params]
