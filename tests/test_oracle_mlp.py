"""Pins for the FP64 MLP oracle of the learned extrapolation: central finite differences,
closed forms and a planted mistake."""
import numpy as np

from oracle import mlp as N


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = N.init(1) + 0.05 * rng.standard_normal(N.NPARAM)
    X = rng.standard_normal((7, 40))
    y = rng.uniform(1, 4, 7)
    _, g = N.loss_and_grad(theta, X, y)
    idx = rng.choice(N.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [N.NPARAM - 1, N.NPARAM - 65, 0, 64 * 40 + 3]])  # b3, w3, W1, b1
    h = 1e-6
    for i in idx:
        e = np.zeros(N.NPARAM)
        e[i] = h
        fd = (N.loss_and_grad(theta + e, X, y)[0] - N.loss_and_grad(theta - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_zero_weights_give_midpoint_step():
    alpha, _ = N.forward(np.zeros(N.NPARAM), np.random.default_rng(1).standard_normal((5, 40)))
    np.testing.assert_array_equal(alpha, 2.5)  # z = 0 -> 1 + 3 * sigmoid(0)


def test_alpha_stays_in_range():
    theta = 30.0 * np.random.default_rng(2).standard_normal(N.NPARAM)
    alpha, _ = N.forward(theta, 10.0 * np.random.default_rng(3).standard_normal((50, 40)))
    assert np.all(alpha >= 1.0) and np.all(alpha <= 4.0)


def test_adam_first_step_is_sign_step():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = N.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-8)


def test_planted_missing_tanh_derivative_is_caught():
    rng = np.random.default_rng(4)
    theta = N.init(5)
    X, y = rng.standard_normal((4, 40)), rng.uniform(1, 4, 4)
    p = N.unpack(theta)
    alpha, c = N.forward(theta, X)
    dz = 2.0 * (alpha - y) / 4 * 3.0 * c["s"] * (1 - c["s"])
    bad_W2 = (np.outer(dz, p["w3"])).T @ c["h1"]  # (1 - h2^2) dropped
    _, g = N.loss_and_grad(theta, X, y)
    good_W2 = N.unpack(g)["W2"]
    assert np.max(np.abs(bad_W2 - good_W2)) > 1e-4 * np.max(np.abs(good_W2))


def test_features_hand_example():
    L = [8.0, 4.0, 1.0]          # decrements ln 2 and ln 4 (most recent first)
    ch = [[1e-2, 1e-3, 1e-4, 1e-6], [1e-1, 1.0, 1e-12, 1e-20]]
    f = N.features(L, ch)
    assert abs(f[0] - np.log10(np.log(4.0)) / 6) < 1e-15
    assert abs(f[1] - np.log10(np.log(2.0)) / 6) < 1e-15
    assert np.all(f[2:8] == 0)
    np.testing.assert_allclose(f[8:12], np.array([-1.0, 0.0, -12.0, -12.0]) / 6, atol=1e-15)
    np.testing.assert_allclose(f[12:16], np.array([-2.0, -3.0, -4.0, -6.0]) / 6, atol=1e-15)
    assert np.all(f[16:] == 0)
