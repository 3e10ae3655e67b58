"""Pins of the surrogate's FP64 oracle: closed-form features and SiLU
derivative, and the analytic gradient against central finite differences."""
import numpy as np

from oracle import ezo_surrogate_oracle as so


def test_features_closed_form():
    q = np.array([[0.0, np.pi / 2, -np.pi]])
    X = so.features(q)
    np.testing.assert_allclose(X[0, :3], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(X[0, 3:6], [1, 0, -1], atol=1e-15)
    assert np.all(X[0, 6:] == 0) and X.shape == (1, 64)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(so.num_params()) * 0.05
    X = so.features(rng.uniform(-3, 3, size=(16, 7)))
    t = rng.uniform(-0.1, 0.3, 16)
    loss, g = so.loss_and_grad(p, X, t)
    idx = np.concatenate([rng.choice(so.num_params() - 1, 60, replace=False), [so.num_params() - 1]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (so.loss_and_grad(pp, X, t)[0] - so.loss_and_grad(pm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd)


def test_silu_derivative_closed_form():
    z = np.linspace(-6, 6, 101)
    s = 1 / (1 + np.exp(-z))
    h = 1e-6
    fd = ((z + h) / (1 + np.exp(-(z + h))) - (z - h) / (1 + np.exp(-(z - h)))) / (2 * h)
    np.testing.assert_allclose(s * (1 + z * (1 - s)), fd, atol=1e-8)
