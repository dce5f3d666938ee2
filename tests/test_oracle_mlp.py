"""Pins of the oracle surrogate network: GELU against its definition's limits and derivative,
backpropagated gradients against central finite differences, and Adam against a hand-computed
first step and convergence on a convex quadratic."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_values_and_derivative():
    z = np.linspace(-6, 6, 241)
    g = mlp.gelu(z)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(g[z > 5], z[z > 5], atol=1e-5) and np.allclose(g[z < -5], 0.0, atol=1e-5)
    # x * standard normal cdf at a point computed by hand: Phi(1) = 0.8413447460685429
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [5, 7, 6, 3]
    W, b = mlp.init_params(sizes, 1)
    b = [rng.normal(0, 0.1, x.shape) for x in b]
    x = rng.normal(0, 1, (9, 5))
    t = rng.normal(0, 1, (9, 3))
    loss, gW, gb = mlp.loss_and_grads(W, b, x, t)
    h = 1e-6
    for l in range(3):
        for idx in [(0, 0), (W[l].shape[0] - 1, W[l].shape[1] - 1), (1, 2)]:
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (mlp.loss_and_grads(Wp, b, x, t)[0] - mlp.loss_and_grads(Wm, b, x, t)[0]) / (2 * h)
            assert gW[l][idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        bp = [v.copy() for v in b]
        bm = [v.copy() for v in b]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (mlp.loss_and_grads(W, bp, x, t)[0] - mlp.loss_and_grads(W, bm, x, t)[0]) / (2 * h)
        assert gb[l][0] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adam_first_step_and_convergence():
    # first step moves every coordinate by -lr * sign(g) (mhat = g, vhat = g^2)
    p = [np.array([1.0, -2.0, 3.0])]
    opt = mlp.Adam(p, lr=0.1, eps=0.0)
    opt.step(p, [np.array([0.5, -4.0, 1e-3])])
    assert np.allclose(p[0], [0.9, -1.9, 2.9], rtol=1e-14)
    # convex quadratic 1/2 |A w - c|^2 converges
    rng = np.random.default_rng(2)
    A = rng.normal(0, 1, (8, 4))
    c = rng.normal(0, 1, 8)
    w = [np.zeros(4)]
    opt = mlp.Adam(w, lr=0.05)
    for _ in range(3000):
        opt.step(w, [A.T @ (A @ w[0] - c)])
    assert np.allclose(w[0], np.linalg.lstsq(A, c, rcond=None)[0], atol=1e-3)
