"""Pins of the FP64 surrogate oracle: a toy network worked by hand, closed forms of the
features, central finite differences of the gradient, and Adam's first step."""
import numpy as np
import pytest

from oracle import mlp as M


def test_features_closed_forms():
    g = M.features([0.0, 0.5, 1.0], [0.0, 0.25, 1.0])
    assert g.shape == (3, 64)
    # u = 0: every sine 0, every cosine 1
    assert np.allclose(g[0, :16], 0.0) and np.allclose(g[0, 16:32], 1.0)
    # u = 1/2: sin(pi k / 2) = 1, 0, -1, 0, ...; cos = 0, -1, 0, 1, ...
    assert np.allclose(g[1, :4], [1, 0, -1, 0], atol=1e-15)
    assert np.allclose(g[1, 16:20], [0, -1, 0, 1], atol=1e-15)
    # u = 1: sines 0, cosines (-1)^k -- the features do not repeat from u = 0 to 1
    assert np.allclose(g[2, :16], 0.0, atol=1e-14)
    assert np.allclose(g[2, 16:32], [(-1) ** k for k in range(1, 17)], atol=1e-14)
    # v = 1/4, k = 2: sin(pi / 2) = 1
    assert g[1, 32 + 1] == pytest.approx(1.0, abs=1e-15)


def test_toy_network_by_hand():
    # Zero every weight except a handful and check the output by hand:
    # h1_0 = relu(g_0 - 2 g_16 + 0.5) with g_0 = sin(pi u), g_16 = cos(pi u);
    # h2_0 = relu(2 h1_0 - 0.25); y = (3 h2_0 + 0.1, -h2_0, 0.2)
    theta = np.zeros(M.N_PARAMS)
    p = M.unpack(theta.copy())
    p["W1"][0, 0] = 1.0
    p["b1"][0] = 0.5
    p["W2"][0, 0] = 2.0
    p["b2"][0] = -0.25
    p["W3"][0, 0] = 3.0
    p["W3"][0, 1] = -1.0
    p["b3"][:] = [0.1, 0.0, 0.2]
    p["W1"][16, 0] = -2.0          # lets unit 0 reach the relu's zero side
    theta = M.pack(p)
    u = np.array([0.5, 0.0, 0.3])
    g = M.features(u, np.zeros(3))
    y, _ = M.forward(theta, g)
    for i, uu in enumerate(u):
        h1 = max(np.sin(np.pi * uu) - 2 * np.cos(np.pi * uu) + 0.5, 0.0)
        h2 = max(2 * h1 - 0.25, 0.0)
        assert np.allclose(y[i], [3 * h2 + 0.1, -h2, 0.2], atol=1e-14)
    # u = 1/2: h1 = 1.5, h2 = 2.75; u = 0: h1 = relu(-1.5) = 0, h2 = 0
    assert np.allclose(y[0], [8.35, -2.75, 0.2], atol=1e-13)
    assert np.allclose(y[1], [0.1, 0.0, 0.2], atol=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.2, M.N_PARAMS)
    u, v = rng.random(20), rng.random(20)
    g = M.features(u, v)
    t = rng.random((20, 3))
    _, grad = M.gradient(theta, g, t)
    idx = rng.choice(M.N_PARAMS, 60, replace=False)
    # include every bias and the last layer
    idx = np.unique(np.concatenate([idx, np.arange(M.N_PARAMS - 195, M.N_PARAMS)]))
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = h
        fd = (M.loss(theta + e, g, t) - M.loss(theta - e, g, t)) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adam_first_step_moves_each_weight_by_lr():
    # With bias correction the first update is lr * g / (|g| + eps) ~ lr * sign(g).
    theta = np.zeros(5)
    grad = np.array([0.5, -2.0, 1e-3, -1e-4, 3.0])
    th, m, v = M.adam_step(theta, np.zeros(5), np.zeros(5), grad, 1, 0.01)
    assert np.allclose(th, -0.01 * np.sign(grad), rtol=1e-4)
    assert np.allclose(m, 0.1 * grad) and np.allclose(v, 0.001 * grad ** 2)


def test_bf16_rounding():
    assert M.bf16_round(1.0) == 1.0
    assert M.bf16_round(1.0 + 2 ** -8) == 1.0              # tie to even
    assert M.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert M.bf16_round(-0.1) == pytest.approx(-0.10009765625, abs=0)
