"""Pins for the threshold-MLP oracle (no GPU).

The oracle's backprop is checked against central finite differences of its
own loss (a different computation: forward passes only), its forward pass
against the closed form the network reduces to when every ReLU is active,
Adam against its first-step identity, and training against a target it must
be able to fit.  A transposed weight, a dropped bias or a missing ReLU mask
fails one of them.
"""
import numpy as np
import pytest

import synth
from oracle import mlp


def _theta(seed, scale=0.4):
    return synth.normal((mlp.N_PARAMS,), seed).astype(np.float64) * scale


def test_layout_is_1281_parameters_and_round_trips():
    assert mlp.N_PARAMS == 32 * 5 + 32 + 32 * 32 + 32 + 32 + 1 == 1281
    th = _theta(11)
    assert np.array_equal(mlp.pack(mlp.unpack(th)), th)
    p = mlp.unpack(np.arange(mlp.N_PARAMS, dtype=np.float64))
    # order: W1 row-major, b1, W2 row-major, b2, W3, b3
    assert p["W1"][1, 0] == 5 and p["b1"][0] == 160 and p["W2"][0, 1] == 193
    assert p["b2"][0] == 1216 and p["W3"][0] == 1248 and p["b3"][0] == 1280


def test_gradient_matches_central_differences():
    th = _theta(12)
    X = synth.uniform((48, mlp.N_IN), 13)
    t = synth.normal((48,), 14)
    _, (_, z1, _, z2, _) = mlp.forward(th, X)
    # keep away from ReLU kinks, where the derivative is not defined
    assert np.abs(z1).min() > 1e-4 and np.abs(z2).min() > 1e-4  # step h moves z by < 1e-5
    L, g = mlp.grad(th, X, t)
    assert L == pytest.approx(mlp.loss(th, X, t), rel=1e-14)
    h = 1e-6
    fd = np.empty_like(th)
    for i in range(mlp.N_PARAMS):
        e = np.zeros_like(th)
        e[i] = h
        fd[i] = (mlp.loss(th + e, X, t) - mlp.loss(th - e, X, t)) / (2 * h)
    scale = np.abs(g).max()
    assert np.abs(fd - g).max() <= 1e-6 * scale


def test_all_active_network_is_the_affine_closed_form():
    """With non-negative weights and inputs every ReLU passes its input, so
    y = W3 (W2 (W1 x + b1) + b2) + b3, and d loss / d b3 = 2 mean(y - t)."""
    th = np.abs(_theta(15))
    X = np.abs(synth.uniform((20, mlp.N_IN), 16))
    t = synth.normal((20,), 17)
    p = mlp.unpack(th)
    want = ((X @ p["W1"].T + p["b1"]) @ p["W2"].T + p["b2"]) @ p["W3"] + p["b3"][0]
    y, _ = mlp.forward(th, X)
    np.testing.assert_allclose(y, want, rtol=1e-13)
    _, g = mlp.grad(th, X, t)
    gp = mlp.unpack(g)
    assert gp["b3"][0] == pytest.approx(2 * np.mean(want - t), rel=1e-12)
    # d loss / d b2_j = sum_s dy_s W3_j  (every unit active)
    np.testing.assert_allclose(gp["b2"], 2 * np.mean(want - t) * p["W3"], rtol=1e-12)


def test_dead_units_get_no_gradient():
    """A hidden unit whose pre-activation is negative on every sample passes
    no gradient to its incoming weights."""
    th = _theta(18)
    p = mlp.unpack(th)
    p["b1"][3] = -1e3
    th = mlp.pack(p)
    X = synth.uniform((30, mlp.N_IN), 19)
    _, g = mlp.grad(th, X, synth.normal((30,), 20))
    gp = mlp.unpack(g)
    assert np.all(gp["W1"][3] == 0) and gp["b1"][3] == 0 and np.all(gp["W2"][:, 3] == 0)


def test_adam_first_step_moves_each_parameter_by_lr():
    """From zero moments, step 1 gives m_hat = g and v_hat = g^2, so each
    parameter moves by lr * g / (|g| + eps)."""
    th = _theta(21)
    g = synth.normal((mlp.N_PARAMS,), 22).astype(np.float64)
    z = np.zeros_like(th)
    lr, eps = 1e-2, 1e-8
    th1, m, v = mlp.adam_step(th, g, z, z, 1, lr, eps=eps)
    np.testing.assert_allclose(th1, th - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_training_fits_a_linear_target():
    X = synth.uniform((512, mlp.N_IN), 23)
    t = 0.3 * X[:, 0] - 0.2 * X[:, 1] + 0.5
    th0 = _theta(24, scale=0.2)
    th, losses = mlp.train(th0, X, t, epochs=60, batch=64, lr=3e-3)
    assert losses[-1] < 2e-3 < losses[0]


def test_coherence_and_features():
    r = synth.normal((1, 50), 25)
    assert mlp.coherence(np.repeat(r, 8, axis=0), axis=0) == pytest.approx(1.0)
    assert mlp.coherence(np.vstack([r, -r]), axis=0) == 0.0
    assert mlp.coherence(np.zeros((4, 4)), axis=0) == 0.0
    # independent zero-mean rows: about 1/sqrt(rows)
    c = mlp.coherence(synth.normal((256, 4096), 26), axis=0)
    assert abs(c - 1 / 16) < 0.01
    x = mlp.features(4096, 120, 248, 0.25, 0.5, "bf16")
    np.testing.assert_allclose(x, [12 / 16, 0.25, 0.5, 0.5, np.log2(120 * 248) / 16])
