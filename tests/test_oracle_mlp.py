"""Pins of the FP64 surrogate oracle (CPU only): analytic gradients against
central finite differences, closed forms of a zero network, the loss at a
zero logit, and the first Adam step."""
import math

import numpy as np
import pytest

from oracle import mlp


def batch(seed=3, B=16):
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.uniform(-1, 1, size=(B, 5))
    t = rng.normal(size=B)
    y = (rng.uniform(size=B) > 0.5).astype(np.float64)
    return z, t, y


def test_gradients_match_central_differences():
    params = mlp.init_params(seed=11)
    z, t, y = batch()
    g = mlp.flatten(mlp.gradients(params, z, t, y, lam=0.7))
    w = mlp.flatten(params)
    rng = np.random.Generator(np.random.PCG64(5))
    idx = rng.choice(w.size, size=300, replace=False)
    # include every bias of the output layer and the first input weights
    idx = np.unique(np.concatenate([idx, np.arange(w.size - 2, w.size), np.arange(0, 5)]))
    h = 1e-6
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (mlp.loss(mlp.unflatten(wp), z, t, y, 0.7) - mlp.loss(mlp.unflatten(wm), z, t, y, 0.7)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1e-3, abs(g[k])) + 1e-10, (k, fd, g[k])


def test_zero_network_closed_form():
    params = [(np.zeros_like(W), np.zeros_like(b)) for W, b in mlp.init_params()]
    z, t, y = batch(B=32)
    out, _ = mlp.forward(params, z)
    assert np.all(out == 0.0)
    assert mlp.loss(params, z, t, y, 1.0) == pytest.approx(np.mean(t ** 2) + math.log(2.0), rel=1e-15)
    g = mlp.gradients(params, z, t, y, 1.0)
    assert g[-1][1][0] == pytest.approx(-2.0 * np.mean(t), rel=1e-14)
    assert g[-1][1][1] == pytest.approx(0.5 - np.mean(y), rel=1e-14, abs=1e-16)
    for dW, db in g[:-1]:  # hidden layers see zero downstream weights
        assert np.all(dW == 0.0) and np.all(db == 0.0)


def test_bce_stable_and_symmetric():
    z = np.array([-800.0, -30.0, 0.0, 30.0, 800.0])
    for y in (0.0, 1.0):
        v = mlp.bce_with_logits(z, y)
        assert np.all(np.isfinite(v)) and np.all(v >= 0.0)
    assert mlp.bce_with_logits(np.array([0.0]), 1.0)[0] == pytest.approx(math.log(2.0), rel=1e-15)
    np.testing.assert_allclose(mlp.bce_with_logits(z, 1.0), mlp.bce_with_logits(-z, 0.0), rtol=1e-15)
    np.testing.assert_allclose(mlp.sigmoid(z) + mlp.sigmoid(-z), 1.0, rtol=1e-15)


def test_adam_first_step_moves_by_lr_times_sign():
    w = np.array([0.3, -1.2, 2.0])
    g = np.array([1e-3, -5.0, 0.0])
    opt = mlp.Adam(3, lr=0.01)
    w1 = opt.step(w, g)
    np.testing.assert_allclose(w1[:2], w[:2] - 0.01 * np.sign(g[:2]), rtol=0, atol=1e-7)
    assert w1[2] == w[2]
