"""Plain FP64 reference of the warm-start network: a multilayer perceptron
5 -> 128 -> 128 -> 128 -> 128 -> 1 with SiLU activations, mean-squared-error loss
and Adam.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): used by the tests to check
the GPU forward pass, gradients and optimiser step.  Written with numpy in double
precision, layer by layer, with no fusion; pinned in tests/test_oracle_mlp.py by
central finite differences of the loss and by closed forms of SiLU.

Parameter layout (shared convention with the GPU library, which stores the same
matrices): W_l is [fan_in, fan_out] row-major, b_l is [fan_out];
z_l = h_{l-1} W_l + b_l, h_l = silu(z_l) for l = 1..4, y = h_4 W_5 + b_5.
"""
from __future__ import annotations

import numpy as np

SIZES = (5, 128, 128, 128, 128, 1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, X):
    """params: list of (W, b); X: [B, 5].  Returns y [B] and the cache."""
    h = np.asarray(X, dtype=np.float64)
    cache = [(h, None)]
    for i, (W, b) in enumerate(params):
        z = h @ W + b
        if i < len(params) - 1:
            h = silu(z)
        else:
            h = z
        cache.append((h, z))
    return h[:, 0], cache


def loss_and_grads(params, X, t):
    """MSE loss mean((y - t)^2) and its gradients w.r.t. every W, b."""
    y, cache = forward(params, X)
    B = len(t)
    r = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    dh = (2.0 / B) * r[:, None]
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, b = params[i]
        h_prev = cache[i][0]
        z = cache[i + 1][1]
        dz = dh if i == len(params) - 1 else dh * silu_grad(z)
        grads[i] = (h_prev.T @ dz, dz.sum(axis=0))
        dh = dz @ W.T
    return loss, grads


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; returns new params, m, v."""
    new_p, new_m, new_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        out = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1 - beta1) * g
            vv = beta2 * vv + (1 - beta2) * g * g
            mhat = mm / (1 - beta1 ** t)
            vhat = vv / (1 - beta2 ** t)
            out.append((p - lr * mhat / (np.sqrt(vhat) + eps), mm, vv))
        new_p.append((out[0][0], out[1][0]))
        new_m.append((out[0][1], out[1][1]))
        new_v.append((out[0][2], out[1][2]))
    return new_p, new_m, new_v


def init_params(seed=1906):
    """He-uniform weights, zero biases (any initialisation serves the tests)."""
    rng = np.random.default_rng(seed)
    params = []
    for fi, fo in zip(SIZES[:-1], SIZES[1:]):
        lim = np.sqrt(6.0 / fi)
        params.append((rng.uniform(-lim, lim, size=(fi, fo)), np.zeros(fo)))
    return params
