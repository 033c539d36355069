"""Pins of the reference MLP (oracle/mlp.py): SiLU and its derivative against
closed forms, every gradient against central finite differences of the loss,
and one Adam step against its definition on a scalar problem."""
import numpy as np
import pytest

from oracle import mlp


def test_silu_closed_forms():
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    z = np.array([-3.0, -0.5, 0.7, 4.0])
    np.testing.assert_allclose(mlp.silu(z), z * 0.5 * (1 + np.tanh(z / 2)), rtol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(mlp.silu_grad(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), rtol=1e-8)
    assert mlp.silu_grad(np.array([0.0]))[0] == pytest.approx(0.5)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(5)
    params = mlp.init_params(seed=3)
    X = rng.normal(size=(7, 5))
    t = rng.normal(size=7)
    loss, grads = mlp.loss_and_grads(params, X, t)
    eps = 1e-6
    for li in range(len(params)):
        for which in (0, 1):
            arr = params[li][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = mlp.loss_and_grads(params, X, t)
                flat[idx] = old - eps
                lm, _ = mlp.loss_and_grads(params, X, t)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                g = grads[li][which].reshape(-1)[idx]
                assert g == pytest.approx(fd, rel=1e-5, abs=1e-9), (li, which, idx)


def test_adam_first_step_moves_by_lr():
    """With bias correction the first Adam step is -lr * sign(g) (|g| >> eps)."""
    W = np.array([[1.0, -2.0]])
    b = np.array([0.5])
    g = [(np.array([[0.3, -4.0]]), np.array([2.0]))]
    z = [(np.zeros_like(W), np.zeros_like(b))]
    p, m, v = mlp.adam_step([(W, b)], g, z, z, t=1, lr=0.01)
    np.testing.assert_allclose(p[0][0], W - 0.01 * np.sign(g[0][0]), rtol=1e-6)
    np.testing.assert_allclose(p[0][1], b - 0.01 * np.sign(g[0][1]), rtol=1e-6)
