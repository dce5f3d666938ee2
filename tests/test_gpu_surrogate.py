"""The surrogate network's tensor-core training and inference kernels against the FP64 oracle.

Weights are set identically on both sides (the oracle uses the BF16-rounded values). The GPU keeps
hidden activations and back-propagated errors in BF16 between layers; the oracle runs the same
storage model (oracle.mlp.bf16_round at every place the kernels store BF16) in FP64. What remains is
the FP32 accumulation of the tensor cores and the rare BF16 rounding that falls the other way
because an FP32 value differs from the FP64 one near a rounding boundary (measured on the GB300:
outputs 2.1e-4, gradients 3e-5 .. 4.2e-4 relative Frobenius). Bound: per-tensor relative Frobenius
error <= 2e-3 and cosine >= 0.99999 for gradients, 2e-3 for outputs (the 1e-2 per tensor that a
BF16 network warrants, with room to spare).
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1709_09763_gb300 import native

pytestmark = pytest.mark.gpu

K, NOBS = 32, 49


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _handle():
    obs = np.full((NOBS, 2), 0.5)
    A = np.random.default_rng(0).normal(0, 1, (1, NOBS, K))
    return native.Handle([4], K, obs, np.zeros(NOBS), 1.0, J=64, linear_A=A, seed=9)


def _target_fn(theta):
    rng = np.random.default_rng(42)
    A = rng.normal(0, 1 / np.sqrt(K), (NOBS, K))
    return np.tanh(theta @ A.T) + 0.3 * (theta[:, :1] ** 2)


def _set_random(h, seed):
    d = h.surrogate_dims()
    W, b = omlp.init_params(d, seed)
    rng = np.random.default_rng(seed + 1)
    b = [rng.normal(0, 0.05, x.shape) for x in b]
    W[0][:, K:] = 0.0
    W[4][NOBS:, :] = 0.0
    b[4][NOBS:] = 0.0
    flat = np.concatenate([np.concatenate([w.ravel(), bb]) for w, bb in zip(W, b)]).astype(np.float32)
    mu = np.concatenate([rng.normal(0, 0.1, NOBS), np.zeros(d[5] - NOBS)])
    sd = np.concatenate([rng.uniform(0.5, 2.0, NOBS), np.ones(d[5] - NOBS)])
    h.surrogate_set(0, flat, np.concatenate([mu, sd]).astype(np.float32))
    return flat, mu.astype(np.float32), sd.astype(np.float32)


def _oracle_params(h, flat):
    """The BF16-rounded weights (what the tensor cores multiply), unpadded, FP64."""
    W, b = h.unflatten(flat)
    Wr = [native.bf16_value(native.bf16_bits(w)).astype(np.float64) for w in W]
    Wr[0] = Wr[0][:, :K]
    Wr[4] = Wr[4][:NOBS, :]
    br = [x.astype(np.float64) for x in b]
    br[4] = br[4][:NOBS]
    return Wr, br


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_forward_matches_oracle():
    h = _handle()
    flat, mu, sd = _set_random(h, 3)
    theta = np.random.default_rng(1).normal(0, 1, (300, K))
    G, _ = h.surrogate_predict(0, theta)
    W, b = _oracle_params(h, flat)
    xr = native.bf16_value(native.bf16_bits(theta)).astype(np.float64)
    z, _ = omlp.forward(W, b, xr, omlp.bf16_round)
    Gref = mu[:NOBS].astype(np.float64) + sd[:NOBS] * z
    print(f"surrogate forward rel err {_rel(G, Gref):.3e}")
    assert _rel(G, Gref) < 2e-3
    assert np.max(np.abs((G - Gref) / sd[:NOBS])) < 0.1 * np.max(np.abs(z))


@pytest.mark.parametrize("n", [512, 3000])
def test_gradients_match_oracle(n):
    """Weight gradients are products over the minibatch (K = n): split over the K chunks when the
    output has few tiles (4 splits at 512; 24 at 3000, the last split one chunk wide and the last
    chunk ragged), partial tiles summed in split order."""
    h = _handle()
    flat, mu, sd = _set_random(h, 5)
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 1, (n, K))
    G = mu[:NOBS] + sd[:NOBS] * _target_fn(theta)
    g, loss = h.surrogate_grads(0, theta, G)
    gW, gb = h.unflatten(g)
    W, b = _oracle_params(h, flat)
    xr = native.bf16_value(native.bf16_bits(theta)).astype(np.float64)
    tz = (G - mu[:NOBS]) / sd[:NOBS]
    lref, rW, rb = omlp.loss_and_grads(W, b, xr, tz, omlp.bf16_round)
    assert loss == pytest.approx(lref, rel=2e-3)
    gW0, gW4, gb4 = gW[0][:, :K], gW[4][:NOBS, :], gb[4][:NOBS]
    pairs = [(gW0, rW[0]), (gW[1], rW[1]), (gW[2], rW[2]), (gW[3], rW[3]), (gW4, rW[4]),
             (gb[0], rb[0]), (gb[3], rb[3]), (gb4, rb[4])]
    errs = [_rel(a, r) for a, r in pairs]
    print("surrogate gradient rel errs " + " ".join(f"{e:.2e}" for e in errs))
    for a, r in pairs:
        assert _rel(a, r) < 2e-3
        cos = np.sum(a * r) / (np.linalg.norm(a) * np.linalg.norm(r))
        assert cos > 0.99999
    # padding receives no gradient
    assert np.all(gW[0][:, K:] == 0) and np.all(gW[4][NOBS:, :] == 0)


def test_training_reduces_loss_and_generalises():
    h = _handle()
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 1, (6000, K))
    G = 0.01 + 0.002 * _target_fn(theta)
    h.surrogate_add_pairs(0, theta, G)
    loss0 = h.surrogate_train(0, 1, 512)
    loss1 = h.surrogate_train(0, 600, 512)
    assert loss1 < 0.1 * loss0
    test = rng.normal(0, 1, (500, K))
    Gt = 0.01 + 0.002 * _target_fn(test)
    Gp, _ = h.surrogate_predict(0, test)
    # relative to the spread of the targets: the trained network explains most of the variance
    assert np.mean((Gp - Gt) ** 2) < 0.1 * np.var(Gt, axis=0).mean()
