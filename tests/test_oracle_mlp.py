"""Pins of the FP64 reference of the learned stand-in's network: gradients against central
finite differences, and the pinball loss's defining property (its minimiser is the quantile).
CPU only."""
import numpy as np

from oracle import mlp


def _problem(rows=6, seed=0):
    rng = np.random.default_rng(seed)
    p = np.concatenate([np.concatenate([rng.normal(0, np.sqrt(2.0 / mlp.DIMS[i]), mlp.DIMS[i] * mlp.DIMS[i + 1]),
                                        rng.normal(0, 0.1, mlp.DIMS[i + 1])]) for i in range(len(mlp.DIMS) - 1)])
    x = rng.normal(size=(rows, 32))
    y = rng.normal(size=(rows, 16))
    tau = rng.uniform(0.05, 0.95, size=(rows, 16))
    mask = (rng.uniform(size=(rows, 16)) < 0.7).astype(float)
    return p, x, y, tau, mask


def test_parameter_count():
    assert mlp.N_PARAMS == 209936


def test_gradient_matches_finite_differences():
    p, x, y, tau, mask = _problem()
    loss, g, _ = mlp.grad(p, x, y, tau, mask)
    rng = np.random.default_rng(1)
    # parameters of every layer, weights and biases
    idx = np.concatenate([rng.integers(0, mlp.N_PARAMS, 30), np.arange(8192, 8192 + 5),
                          np.arange(mlp.N_PARAMS - 16, mlp.N_PARAMS)])
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (mlp.pinball(mlp.forward(pp, x)[1], y, tau, mask) - mlp.pinball(mlp.forward(pm, x)[1], y, tau, mask)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_pinball_minimiser_is_the_quantile():
    rng = np.random.default_rng(2)
    y = rng.exponential(size=4001)
    for tau in (0.1, 0.5, 0.9):
        grid = np.linspace(0, 5, 5001)
        losses = [np.mean((y - c) * (tau - (y - c < 0))) for c in grid]
        assert abs(grid[int(np.argmin(losses))] - np.quantile(y, tau)) < 2e-3


def test_bf16_rounding():
    a = np.array([1.0, 1.00390625, 1.0 + 2 ** -9, -3.14159, 1e-3], dtype=np.float64)
    r = mlp.bf16(a)
    assert r[0] == 1.0 and r[1] == 1.0                           # halfway: ties to the even significand
    assert np.all(np.abs(r - a) <= np.abs(a) * 2 ** -8)
