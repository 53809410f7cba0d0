"""FP64 oracle of the surrogate network that seeds the non-LTE iteration.

TEST INFRASTRUCTURE ONLY.  The paper has no learned component: this restates, in
plain numpy, the small fully connected network the GPU trains and runs --
x -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> W3 h2 + b3 (6 -> 64 -> 64 -> 3) with
input standardisation, a mean-squared-error loss, the textbook backward pass
(chain rule, one layer at a time) and the Adam update (Kingma & Ba 2015,
bias-corrected moments).  The parameter vector is flattened in the order
W1, b1, W2, b2, W3, b3 with W stored [out][in] row-major.
"""
from __future__ import annotations

import numpy as np


def sizes(n_in=6, n_hidden=64, n_out=3):
    return [(n_hidden, n_in), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_out, n_hidden),
            (n_out,)]


def unflatten(theta, n_in=6, n_hidden=64, n_out=3):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for shp in sizes(n_in, n_hidden, n_out):
        k = int(np.prod(shp))
        out.append(theta[o:o + k].reshape(shp))
        o += k
    assert o == theta.size
    return out


def flatten(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params])


def forward(theta, X, mean, std, n_hidden=64, n_out=3):
    """Network output [B][n_out] and the activations the backward pass needs."""
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unflatten(theta, X.shape[1], n_hidden, n_out)
    xn = (X - mean) / std
    h1 = np.tanh(xn @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ W3.T + b3
    return y, (xn, h1, h2)


def loss_and_grad(theta, X, Y, mean, std, n_hidden=64, n_out=3):
    """Mean over samples and outputs of (y - Y)^2, and its gradient in flattened order."""
    Y = np.asarray(Y, dtype=np.float64)
    B = Y.shape[0]
    W1, b1, W2, b2, W3, b3 = unflatten(theta, np.asarray(X).shape[1], n_hidden, n_out)
    y, (xn, h1, h2) = forward(theta, X, mean, std, n_hidden, n_out)
    r = y - Y
    loss = float(np.mean(r * r))
    dy = 2.0 * r / (B * n_out)                       # d loss / d y
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dh2 = (dy @ W3) * (1.0 - h2 * h2)               # through tanh
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (1.0 - h1 * h1)
    gW1 = dh1.T @ xn
    gb1 = dh1.sum(axis=0)
    return loss, flatten([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new theta, m, v."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def round_bf16(a):
    """Round-to-nearest-even to bfloat16 (the weights the GPU multiplies with)."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
