"""Pins for the oracle's SIREN surrogate: analytic gradients against central
finite differences, Adam against its closed form on a quadratic."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("omega0", [1.0, 30.0])
def test_gradient_matches_finite_differences(omega0):
    rng = np.random.default_rng(0)
    sizes = mlp.layer_sizes(5, 6, 4, 2)
    p = rng.uniform(-0.5, 0.5, mlp.n_params(sizes)) / (omega0 if omega0 > 1 else 1.0)
    X = rng.uniform(-1, 1, (7, 5))
    T = rng.standard_normal((7, 4))
    Y, cache = mlp.forward(p, sizes, X, omega0)
    g = mlp.backward(p, sizes, cache, Y, T, omega0)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(mlp.forward(p + e, sizes, X, omega0)[0], T)
                 - mlp.loss(mlp.forward(p - e, sizes, X, omega0)[0], T)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_layer_layout_and_count():
    sizes = mlp.layer_sizes(5, 128, 4, 16)
    assert sizes == [5, 128, 128, 128, 128, 32]
    assert mlp.n_params(sizes) == 5 * 128 + 128 + 3 * (128 * 128 + 128) + 128 * 32 + 32
    p = np.arange(mlp.n_params(sizes), dtype=np.float64)
    (W1, b1) = mlp.unpack(p, sizes)[0]
    assert W1.shape == (128, 5) and W1[0, 1] == 1 and b1[0] == 640


def test_adam_first_step_moves_by_lr_times_sign():
    # with bias correction, the first Adam step is -lr * g / (|g| + eps)
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_converges_on_a_quadratic():
    p = np.array([3.0, -1.0])
    m = v = np.zeros(2)
    for t in range(1, 3001):
        p, m, v = mlp.adam_step(p, 2 * p, m, v, t, 0.05)
    assert np.all(np.abs(p) < 1e-3)
