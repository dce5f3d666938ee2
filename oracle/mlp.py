"""Surrogate network theta -> G_l(theta) and its training (oracle, FP64).

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle; never imported by the product library.

The paper has no surrogate; the library adds one as the first stage of a delayed-acceptance pCN
move (Christen & Fox 2005), so the exact potential still decides every accepted move. Network:
x -> GELU(W1 x + b1) -> GELU(W2 . + b2) -> ... -> W_L . + b_L, with the exact GELU
g(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2. It predicts standardised observations
z = (G - mu) / s (per-output mean mu and standard deviation s of the training targets); the
loss is the mean squared error over batch and outputs. Adam (Kingma & Ba 2015):
m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2, w <- w - lr mhat / (sqrt(vhat) + eps) with
mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).

Storage model (optional `store` argument of forward and loss_and_grads): a network that keeps its
activations and back-propagated errors in a narrow format rounds them where it writes them. With
store = bf16_round the oracle rounds, in the same places, every hidden activation GELU(z) and every
error signal dL/dz (the output error 2 (out - target) / n and each hidden dL/dz after the GELU
derivative); pre-activations z, products and sums stay FP64. store = None is the exact network.
"""
import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def bf16_round(x):
    """x rounded to FP32 (nearest) and then to BF16 (8 significant bits, nearest, ties to even),
    returned as FP64: the value a BF16 store of an FP32 result holds."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) << np.uint64(16)
    return (u & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(sizes, seed):
    """He-style normal init, weights W[l] of shape (out, in), zero biases."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for i in range(len(sizes) - 1):
        W.append(rng.normal(0.0, math.sqrt(2.0 / sizes[i]), (sizes[i + 1], sizes[i])))
        b.append(np.zeros(sizes[i + 1]))
    return W, b


def _keep(v):
    return v


def forward(W, b, x, store=None):
    """Returns the output and the cache (inputs of each layer, pre-activations). `store` rounds
    each hidden activation (storage model above)."""
    store = store or _keep
    acts, pres = [np.asarray(x, dtype=np.float64)], []
    h = acts[0]
    for l in range(len(W)):
        z = h @ W[l].T + b[l]
        pres.append(z)
        h = store(gelu(z)) if l < len(W) - 1 else z
        acts.append(h)
    return h, (acts, pres)


def loss_and_grads(W, b, x, target, store=None):
    """Mean squared error over all entries and its gradients (backpropagation). `store` rounds
    the activations and the error signals dL/dz (storage model above)."""
    store = store or _keep
    out, (acts, pres) = forward(W, b, x, store)
    n = out.size
    diff = out - target
    loss = float(np.sum(diff * diff) / n)
    d = store(2.0 * diff / n)
    gW, gb = [None] * len(W), [None] * len(W)
    for l in range(len(W) - 1, -1, -1):
        if l < len(W) - 1:
            d = store(d * gelu_grad(pres[l]))
        gW[l] = d.T @ acts[l]
        gb[l] = d.sum(axis=0)
        d = d @ W[l]
    return loss, gW, gb


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.b1
            m += (1.0 - self.b1) * g
            v *= self.b2
            v += (1.0 - self.b2) * g * g
            p -= self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps)
