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


def test_bf16_round_against_hand_values_and_torch():
    """The storage model's rounding: 8 significant bits, nearest, ties to even, checked on
    hand-computed values and against torch's float32 -> bfloat16 conversion (a library routine)."""
    torch = pytest.importorskip("torch")
    e = 2.0 ** -8
    cases = {1.0: 1.0, 1.0 + e: 1.0, 1.0 + 3 * e: 1.0 + 4 * e, 1.0 + 1.5 * e: 1.0 + 2 * e,
             -(1.0 + 3 * e): -(1.0 + 4 * e), 3.0: 3.0, 0.0: 0.0, 2.0 ** -130: 2.0 ** -130}
    for x, want in cases.items():
        assert mlp.bf16_round(np.array([x]))[0] == want
    x = np.random.default_rng(3).normal(0, 1, 20000) * np.exp(np.random.default_rng(4).normal(0, 8, 20000))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_storage_model_rounds_only_stored_values():
    """With store = bf16_round every hidden activation is a BF16 value, the pre-activations are
    the exact affine maps of the stored inputs, and the gradients stay within the first-order
    effect of relative perturbations of 2^-9 per stored value (a few per cent for a four-layer net)."""
    rng = np.random.default_rng(5)
    sizes = [6, 16, 16, 16, 4]
    W, b = mlp.init_params(sizes, 2)
    x = rng.normal(0, 1, (32, 6))
    t = rng.normal(0, 1, (32, 4))
    out, (acts, pres) = mlp.forward(W, b, x, mlp.bf16_round)
    for l in range(1, len(W)):
        assert np.array_equal(mlp.bf16_round(acts[l]), acts[l])
        assert np.allclose(pres[l], acts[l] @ W[l].T + b[l], rtol=0, atol=0)
    l0, gW0, gb0 = mlp.loss_and_grads(W, b, x, t)
    l1, gW1, gb1 = mlp.loss_and_grads(W, b, x, t, mlp.bf16_round)
    assert abs(l1 - l0) < 2e-2 * l0
    for a, r in zip(gW1 + gb1, gW0 + gb0):
        assert np.linalg.norm(a - r) < 5e-2 * np.linalg.norm(r)
    # rounding the stored values is not the identity (the model is active)
    assert not np.array_equal(gW1[0], gW0[0])
