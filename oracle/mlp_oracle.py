"""FP64 CPU reference of the pose-dynamics MLP surrogate.

TEST INFRASTRUCTURE ONLY (tests and the CPU baseline may run it; the product
path never imports it).  A plain multilayer perceptron written out step by
step in numpy float64:

    a_0 = x
    z_l = a_{l-1} W_l^T + b_l,   a_l = SiLU(z_l) = z_l * sigmoid(z_l)   (l < L)
    y   = a_{L-1} W_L^T + b_L                                            (linear head)

with W_l of shape (out_l, in_l).  The reverse sweep is the chain rule on the
same steps:
    dz_L = dy;  dW_l = dz_l^T a_{l-1};  db_l = sum over rows of dz_l;
    da_{l-1} = dz_l W_l;  dz_{l-1} = da_{l-1} * SiLU'(z_{l-1}),
    SiLU'(z) = s (1 + z (1 - s)),  s = sigmoid(z).
Pinned by tests/test_oracle_mlp.py (central finite differences, a linear
special case, and torch.nn reference layers).
"""
from __future__ import annotations

import numpy as np


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(params, x):
    """params: list of (W (out, in), b (out,)).  Returns y and the cache
    (inputs a_{l-1} and pre-activations z_l of every layer)."""
    a = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        z = a @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        cache.append((a, z))
        a = silu(z) if l < len(params) - 1 else z
    return a, cache


def backward(params, cache, dy):
    """Gradients of sum(dy * y): ([(dW_l, db_l)], dx)."""
    grads = [None] * len(params)
    dz = np.asarray(dy, dtype=np.float64)
    for l in range(len(params) - 1, -1, -1):
        a_in, _ = cache[l]
        W = np.asarray(params[l][0], np.float64)
        grads[l] = (dz.T @ a_in, dz.sum(0))
        da = dz @ W
        if l > 0:
            dz = da * silu_grad(cache[l - 1][1])
    return grads, da

