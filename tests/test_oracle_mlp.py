"""Pins of the MLP oracle (learned smoother parameters): gradient against central
finite differences, Adam's first-step property."""
import numpy as np

from oracle import mlp


def _data(B=7, seed=1):
    g = np.random.default_rng(seed)
    return g.standard_normal((B, mlp.IN)), g.standard_normal((B, mlp.OUT)), g.uniform(0.5, 2.0, B)


def test_parameter_count():
    assert mlp.NPARAM == 6 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2 == 4738


def test_gradient_matches_finite_differences():
    theta = mlp.init(3) + 0.05 * np.random.default_rng(2).standard_normal(mlp.NPARAM)
    x, t, w = _data()
    g = mlp.grad(theta, x, t, w)
    rng = np.random.default_rng(4)
    idx = np.concatenate([np.arange(0, 6), rng.choice(mlp.NPARAM, 60, replace=False),
                          np.arange(mlp.NPARAM - 4, mlp.NPARAM)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss(theta + e, x, t, w) - mlp.loss(theta - e, x, t, w)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_loss_definition():
    theta = mlp.init(5)
    x, t, w = _data(B=3)
    y, _, _ = mlp.forward(theta, x)
    ref = sum(w[b] * sum((y[b, o] - t[b, o]) ** 2 for o in range(2)) for b in range(3)) / 3
    assert abs(mlp.loss(theta, x, t, w) - ref) < 1e-12


def test_adam_first_step_moves_by_lr_times_sign():
    # with bias correction, step 1 gives m_hat / sqrt(v_hat) = g / |g|
    theta = np.zeros(5)
    g = np.array([3.0, -0.5, 1e-3, -7.0, 2.0])
    new, m, v = mlp.adam(theta, g, np.zeros(5), np.zeros(5), 1, lr=0.01, eps=0.0)
    assert np.allclose(new, -0.01 * np.sign(g), rtol=1e-12)
