"""Posterior moments of a K = 2 FEM inverse problem by brute-force quadrature (oracle only).

The posterior of Eq. BayesBIP with the discretised potential on the finest level (Sec. 2.2) is
pi(theta) ~ exp(-Phi_h(theta)) N(theta; 0, I_2). Its mean and covariance are integrals over R^2;
with two KL terms they are computed directly: a coarse grid locates the mass, then a
trapezoid grid of n x n points over mode +- 8 standard deviations (the prior density included)
gives the moments; two grid sizes are compared and the difference is stored as the quadrature
error. Forward model: the oracle's P1 FEM on 1/h = 16, observations on the 3 x 3 grid
(i/4, j/4), sigma = 5 % of the largest observation, separable exponential KL with correlation
length 0.3. Data: theta_true = (0.8, -0.5) (seeded noise 4242).

Run:  python tests/golden/make_quadrature.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np                                     # noqa: E402

from oracle import forward as ofwd                     # noqa: E402
from paper_1709_09763_gb300 import workloads as wl     # noqa: E402

N, K, LC = 16, 2, 0.3
OBS = wl.obs_grid(3)
THETA_TRUE = np.array([0.8, -0.5])


def setup():
    lv = ofwd.Level(N, LC, 1.0, K, OBS)
    G = lv.G(THETA_TRUE)
    sigma = 0.05 * np.abs(G).max()
    y = G + sigma * wl.standard_normals((OBS.shape[0],), 4242)
    return lv, y, sigma


def log_post(lv, y, sigma, pts):
    G = lv.G_batch(pts)
    return -ofwd.potential(G, y, sigma) - 0.5 * np.sum(pts * pts, axis=1)


def moments(lv, y, sigma, center, half, n):
    a = np.linspace(center[0] - half[0], center[0] + half[0], n)
    b = np.linspace(center[1] - half[1], center[1] + half[1], n)
    A, B = np.meshgrid(a, b, indexing="ij")
    pts = np.stack([A.ravel(), B.ravel()], axis=1)
    lp = log_post(lv, y, sigma, pts)
    w = np.exp(lp - lp.max()).reshape(n, n)
    wa = np.ones(n); wa[0] = wa[-1] = 0.5
    W = w * wa[:, None] * wa[None, :]
    Z = W.sum()
    m = np.array([(W * A).sum(), (W * B).sum()]) / Z
    v = np.array([(W * (A - m[0]) ** 2).sum(), (W * (B - m[1]) ** 2).sum()]) / Z
    c = (W * (A - m[0]) * (B - m[1])).sum() / Z
    return m, v, c


if __name__ == "__main__":
    lv, y, sigma = setup()
    m0, v0, _ = moments(lv, y, sigma, np.zeros(2), np.array([4.0, 4.0]), 61)
    sd = np.sqrt(v0)
    half = 8.0 * sd
    m1, v1, c1 = moments(lv, y, sigma, m0, half, 81)
    m2, v2, c2 = moments(lv, y, sigma, m0, half, 121)
    out = dict(inv_h=N, K=K, corr_len=LC, obs=OBS.tolist(), theta_true=THETA_TRUE.tolist(), y=y.tolist(),
               sigma=float(sigma), mean=m2.tolist(), var=v2.tolist(), cov01=float(c2),
               quad_err_mean=np.abs(m2 - m1).tolist(), quad_err_var=np.abs(v2 - v1).tolist())
    with open(os.path.join(HERE, "quad_k2_h16.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["mean"], out["var"], out["quad_err_mean"], out["quad_err_var"])
