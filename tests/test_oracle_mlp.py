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


def _toy_theta():
    p = M.unpack(np.zeros(M.N_PARAMS))
    p["W1"][0, 0] = 1.0
    p["W1"][16, 0] = -2.0
    p["b1"][0] = 0.5
    p["W2"][0, 0] = 2.0
    p["b2"][0] = -0.25
    p["W3"][0, 0] = 3.0
    p["W3"][0, 1] = -1.0
    p["b3"][:] = [0.1, 0.0, 0.2]
    return M.pack(p)


def test_c_network_toy_by_hand():
    # the C statement of the network on the hand-worked toy: u = 1/2 gives h1 = 1.5,
    # h2 = 2.75, y = (8.35, -2.75, 0.2); u = 0 gives y = b3
    from oracle import oracle as O
    y = O.mlp_forward(_toy_theta(), [0.5, 0.0], [0.0, 0.0], bf16=False)
    assert np.allclose(y[0], [8.35, -2.75, 0.2], atol=1e-13)
    assert np.allclose(y[1], [0.1, 0.0, 0.2], atol=1e-15)


def test_c_network_bf16_rounding_points():
    # with bf16 the C network rounds the weights: 1 + 2^-9 rounds to 1 (ties to even),
    # so W1[0,0] = 1 + 2^-9 behaves as 1; at u = 1/2 the features (1 and 0) are exact
    from oracle import oracle as O
    th = _toy_theta()
    th[0] = 1.0 + 2.0 ** -9
    exact = O.mlp_forward(th, [0.5], [0.0], bf16=False)[0]
    rounded = O.mlp_forward(th, [0.5], [0.0], bf16=True)[0]
    assert np.allclose(rounded, [8.35, -2.75, 0.2], atol=1e-12)
    # FP64: h1 = 1.5 + 2^-9, h2 = 2.75 + 2^-8, y0 = 8.35 + 3 * 2^-8
    assert exact[0] == pytest.approx(8.35 + 3 * 2.0 ** -8, abs=1e-12)
    # a hidden value of 2.75 + 2^-8 is not a bf16 number: it rounds to 2.75
    assert M.bf16_round(np.array([2.75 + 2.0 ** -8]))[0] == 2.75


def test_constant_surrogate_equals_constant_node():
    # a surrogate with every weight 0 outputs clamp(b3): the material must then shade as
    # the same network with the cacheable node replaced by that constant (plain
    # evaluation, another code path), and the node is neither probed nor inserted
    from oracle import oracle as O
    from paper_2305_07238_gb300 import workload as W
    mats = W.surrogate_materials(1, 40, 60, seed=3)
    mat = mats[0]
    _, roots = O.analyze(mat)
    assert len(roots) == 1
    node = int(roots[0])
    th = np.zeros(M.N_PARAMS)
    th[8512:8515] = [0.25, 1.7, -0.3]
    c = O.Cache(mats, 64, 4)
    c.set_surrogate(0, node, th, bf16=True)
    pts = W.points_uniform(200, seed=4, n_mats=1)
    r = c.run_batch(pts)
    alt = mat.copy()
    alt[node]["op"] = W.OP_CONST
    alt[node]["inp"] = -1
    alt[node]["fp"][:3] = [0.25, 1.0, 0.0]
    for i in range(0, 200, 17):
        sp = [pts[k][i] for k in ("u", "v", "px", "py", "pz", "nx", "ny", "nz")]
        want = O.eval_point_nocache(alt, sp)
        assert np.allclose(r["rgb"][:, i], want, atol=1e-12)
    s = c.stats()
    assert s["lookups"] == 0 and s["candidates"] == 0 and s["inserted"] == 0
    assert not r["hits"].any()
