"""Pins of the warm-start network oracle (oracle/mlp.py) against facts that do
not come from the oracle itself: central finite differences of the loss,
closed forms of the first Adam steps, a planted rotation for Procrustes and a
planted angle for the principal-angle routine."""
import numpy as np
import pytest

from oracle import mlp

SIZES = [5, 7, 6, 3]


def _problem(seed=0, B=4):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.param_count(SIZES)) * 0.5
    X = rng.standard_normal((B, SIZES[0]))
    T = rng.standard_normal((B, SIZES[-1]))
    return p, X, T


def test_param_layout():
    p = np.arange(mlp.param_count(SIZES), dtype=float)
    layers = mlp.unpack(p, SIZES)
    assert [W.shape for W, _ in layers] == [(7, 5), (6, 7), (3, 6)]
    assert layers[0][1][0] == 35.0 and layers[1][0][0, 0] == 42.0
    with pytest.raises(ValueError):
        mlp.unpack(p[:-1], SIZES)


def test_gradient_matches_central_differences():
    p, X, T = _problem()
    loss, g = mlp.backward(p, SIZES, X, T)
    assert loss == pytest.approx(mlp.mse(mlp.forward(p, SIZES, X)[0], T), rel=1e-15)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.mse(mlp.forward(p + e, SIZES, X)[0], T) - mlp.mse(mlp.forward(p - e, SIZES, X)[0], T)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-8 * max(1.0, np.max(np.abs(g)))


def test_single_linear_layer_gradient_closed_form():
    # one linear layer: L = |X W^T + b - T|^2 / (B d), dL/dW = 2 (Y - T)^T X / (B d)
    rng = np.random.default_rng(3)
    sizes = [4, 2]
    W = rng.standard_normal((2, 4))
    b = rng.standard_normal(2)
    X = rng.standard_normal((5, 4))
    T = rng.standard_normal((5, 2))
    _, g = mlp.backward(np.concatenate([W.ravel(), b]), sizes, X, T)
    R = X @ W.T + b - T
    assert np.allclose(g[:8].reshape(2, 4), 2.0 * R.T @ X / 10.0, rtol=1e-13)
    assert np.allclose(g[8:], 2.0 * R.sum(0) / 10.0, rtol=1e-13)


def test_adam_first_steps_closed_form():
    # with a constant gradient g the bias-corrected moments are g and g^2, so
    # every step moves each parameter by lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 1e-2, 1e-8
    for t in (1, 2, 3):
        p_new, m, v = mlp.adam_step(p, g, m, v, t, lr, eps=eps)
        assert np.allclose(p_new - p, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
        p = p_new


def test_adam_descends_on_quadratic():
    # f(p) = |p - c|^2 / 2: Adam with a small rate moves every coordinate toward c
    c = np.array([1.0, -3.0, 0.5])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 2001):
        p, m, v = mlp.adam_step(p, p - c, m, v, t, 1e-2)
    assert np.allclose(p, c, atol=1e-3)


def test_procrustes_recovers_planted_rotation():
    rng = np.random.default_rng(5)
    Xr = rng.standard_normal((40, 6))
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    X = Xr @ Q.T
    assert np.allclose(mlp.procrustes(X, Xr), Xr, atol=1e-12)


def test_max_angle_planted():
    a = 0.37
    X = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    Y = np.array([[1.0, 0.0], [0.0, np.cos(a)], [0.0, np.sin(a)]])
    assert mlp.max_angle(X, Y) == pytest.approx(a, abs=1e-12)
    assert mlp.max_angle(X, X @ np.array([[2.0, 1.0], [0.0, 3.0]])) == pytest.approx(0.0, abs=1e-7)
