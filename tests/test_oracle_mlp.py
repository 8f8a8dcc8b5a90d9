"""Pins of the FP64 MLP oracle (no GPU): gradients against central finite
differences of the loss, Adam against its closed form, feature periodicity,
GELU against its definition's limits, bf16 rounding, SplitMix64 reference values."""
import numpy as np

from oracle import mlp


def test_features_periodic_and_bounded():
    rng = np.random.default_rng(0)
    x = rng.random((50, 3))
    X0 = mlp.features(x, 0.3, 0.1)
    for shift in ((1, 0, 0), (0, -1, 0), (0, 0, 2)):
        X1 = mlp.features(x + np.array(shift), 0.3, 0.1)
        assert np.allclose(X0, X1, atol=1e-12)
    s, c = X0[:, 0:32:2], X0[:, 1:32:2]
    assert np.allclose(s * s + c * c, 1.0)
    assert np.all(X0[:, 34:] == 0)


def test_gelu_limits():
    z = np.array([-30.0, -1.0, 0.0, 1.0, 30.0])
    g = mlp.gelu(z)
    assert abs(g[0]) < 1e-12 and g[2] == 0.0 and abs(g[4] - 30.0) < 1e-12
    h = 1e-6
    assert np.allclose(mlp.gelu_prime(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(3)
    X = mlp.features(rng.random((24, 3)), 0.4, rng.random(24) * 0.2)
    T = rng.standard_normal((24, 4)) * 0.1
    loss, g = mlp.loss_and_grad(theta, X, T)
    # probe a spread of parameters of every layer (padded ones must have 0 gradient)
    sizes = mlp.param_sizes()
    offs = np.cumsum([0] + [fo * fi + fo for fo, fi in sizes])
    picks = []
    for li, (fo, fi) in enumerate(sizes):
        o = offs[li]
        picks += [o + 0, o + 5 * fi + 7, o + (fo - 1) * fi + min(fi - 1, 33), o + fo * fi + 3]
    picks += [offs[4] + 5 * 128 + 2]  # W5 padded output row: gradient 0
    h = 1e-6
    for p in picks:
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (mlp.loss_and_grad(tp, X, T)[0] - mlp.loss_and_grad(tm, X, T)[0]) / (2 * h)
        if p == picks[-1]:
            assert g[p] == 0.0
            continue
        assert abs(fd - g[p]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (p, fd, g[p])


def test_adam_closed_form():
    # constant gradient g: after t steps, m_hat = g and v_hat = g^2 exactly, so each
    # step moves theta by lr * g / (|g| + eps)
    theta = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    for t in range(1, 6):
        theta, m, v = mlp.adam_step(theta, g, m, v, t, lr=0.01)
    step = 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(theta, np.array([1.0, -2.0]) - 5 * step, rtol=0, atol=1e-12)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 1e-3])
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # tie -> even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] - (-3.140625)) < 1e-12
    assert abs(r[4] - 1e-3) / 1e-3 < 2 ** -8


def test_splitmix64_reference():
    # first outputs of SplitMix64 seeded with 0 (state x advanced by the golden gamma)
    assert int(mlp.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    idx = mlp.batch_indices(7, 3, 1000, 97)
    assert idx.min() >= 0 and idx.max() < 97 and len(np.unique(idx)) > 90
