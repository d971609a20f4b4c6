"""Pins for the fp64 schedule-MLP oracle (no GPU).

The backward pass is checked against central finite differences of the loss
(an independent numerical definition of the gradient), against closed forms
for degenerate networks, and Adam against its closed-form first steps.
"""
import numpy as np

from oracle import mlp


def _rand_params(rng, scale=0.5):
    return rng.normal(0, scale, size=mlp.N_PARAMS)


def test_param_count_and_packing():
    assert mlp.N_PARAMS == 32 * 5 + 32 + 32 * 32 + 32 + 8 * 32 + 8 == 1512
    rng = np.random.default_rng(0)
    p = _rand_params(rng)
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)
    P = mlp.unpack(p)
    assert P["W1"][0, 1] == p[1] and P["b1"][0] == p[160] and P["b3"][7] == p[-1]


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    for trial in range(3):
        p = _rand_params(rng)
        B = 7
        X = rng.uniform(0, 1, size=(B, 5))
        act = rng.integers(0, 8, size=B)
        t = rng.normal(size=B)
        L, g = mlp.backward(p, X, act, t)
        assert abs(L - mlp.loss(p, X, act, t)) < 1e-12
        h = 1e-6
        for i in rng.choice(mlp.N_PARAMS, size=120, replace=False):
            e = np.zeros_like(p)
            e[i] = h
            fd = (mlp.loss(p + e, X, act, t) - mlp.loss(p - e, X, act, t)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (trial, i, fd, g[i])


def test_zero_network_closed_forms():
    p = np.zeros(mlp.N_PARAMS)
    P = mlp.unpack(p)
    P["b3"][:] = np.arange(8) * 0.5
    p = mlp.pack(P)
    X = np.random.default_rng(2).uniform(size=(5, 5))
    y, _ = mlp.forward(p, X)
    assert np.allclose(y, np.tile(np.arange(8) * 0.5, (5, 1)), atol=0, rtol=0)
    act = np.array([0, 3, 3, 7, 1])
    t = np.array([1.0, 0.0, 2.0, 3.5, -1.0])
    L, g = mlp.backward(p, X, act, t)
    sel = np.arange(8)[act] * 0.5
    assert abs(L - np.mean((sel - t) ** 2)) < 1e-15
    G = mlp.unpack(g)
    want_b3 = np.zeros(8)
    for a, s, tt in zip(act, sel, t):
        want_b3[a] += 2 * (s - tt) / 5
    assert np.allclose(G["b3"], want_b3, rtol=0, atol=1e-15)
    # hidden activations are all zero -> every other gradient is exactly zero
    for k in ("W1", "b1", "W2", "b2", "W3"):
        assert np.all(G[k] == 0)


def test_dead_relu_blocks_first_layer_gradient():
    rng = np.random.default_rng(3)
    P = mlp.unpack(_rand_params(rng))
    P["W1"][:] = -np.abs(P["W1"])
    P["b1"][:] = -1.0          # z1 < 0 for inputs in [0,1]
    p = mlp.pack(P)
    X = rng.uniform(0, 1, size=(4, 5))
    _, g = mlp.backward(p, X, [1, 2, 3, 4], [0, 0, 0, 0])
    G = mlp.unpack(g)
    assert np.all(G["W1"] == 0) and np.all(G["b1"] == 0)


def test_adam_closed_form_first_steps():
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-2, 1e-8
    p1, m, v = mlp.adam_step(p0, g, m, v, 1, lr=lr, eps=eps)
    # first step: m_hat = g, v_hat = g^2
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    # constant gradient: bias correction keeps m_hat = g, v_hat = g^2 exactly
    p2, m, v = mlp.adam_step(p1, g, m, v, 2, lr=lr, eps=eps)
    assert np.allclose(p2, p1 - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_adam_moment_decay_under_varying_gradients():
    """Adam's moment decay rates (Kingma & Ba 2015, Algorithm 1) pinned by
    hand-derived values.  A constant gradient hides beta1 and beta2 (the
    bias-corrected moments equal g and g^2 for any betas), so this uses
    g = 1, 3, -2 with beta1 = 0.5 and beta2 = 0.75.  Unrolling the moment
    recursions gives the bias-corrected moments as weighted means:
      m_hat_t = sum_i beta1^(t-i) g_i / sum_i beta1^(t-i)
      v_hat_t = sum_i beta2^(t-i) g_i^2 / sum_i beta2^(t-i)
    which for these numbers are, by hand:
      t = 1: m_hat = 1,     v_hat = 1
      t = 2: m_hat = 7/3,   v_hat = 39/7
      t = 3: m_hat = -1/7,  v_hat = 181/37
    and raw moments after step 3: m = 0.5 * (-0.25) = -0.125,
    v = 0.25 * (181/16) = 2.828125.  Swapping the betas gives
    m_hat_2 = 15/7 instead of 7/3, so a swap fails this test."""
    p0 = np.array([0.3])
    m = np.zeros(1)
    v = np.zeros(1)
    lr = 0.1
    steps = [(1.0, 1.0, 1.0), (3.0, 7.0 / 3.0, 39.0 / 7.0), (-2.0, -1.0 / 7.0, 181.0 / 37.0)]
    p = p0
    for t, (g, mh, vh) in enumerate(steps, start=1):
        p_next, m, v = mlp.adam_step(p, np.array([g]), m, v, t, lr=lr, beta1=0.5, beta2=0.75,
                                     eps=0.0)
        assert np.allclose(p_next, p - lr * mh / np.sqrt(vh), rtol=1e-13, atol=0), t
        p = p_next
    assert np.isclose(m[0], -0.125, rtol=1e-13) and np.isclose(v[0], 2.828125, rtol=1e-13)


def test_features_closed_form():
    X = mlp.features([1, 0, 3], [3, 0, 21], [0, 1, 3], [1000, 0, 3000])
    assert np.allclose(X[0], [1 / 24, 2 / 32, 2 ** 0 * np.log2(4) / 8, 0, 1 / 16])
    assert np.allclose(X[1], [0, 0, 0, 1 / 24, 0])
    assert np.allclose(X[2], [2 / 24, np.log2(22) / 32, 3 / 8, 2 / 24, 2 / 16])
    # the round index saturates at 2^14 rounds (log2(1 + 2^14) / 24)
    Y = mlp.features([1, 1], [2, 2], [2 ** 14, 10 ** 7], [0, 0])
    assert np.isclose(Y[0, 3], np.log2(1 + 2 ** 14) / 24) and Y[1, 3] == Y[0, 3]
