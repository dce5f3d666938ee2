"""Truncated Karhunen-Loeve expansion of the prior log-diffusion field (oracle).

TEST INFRASTRUCTURE ONLY: this module is part of the FP64 CPU oracle. Only the
tests, the smoke check and the benchmark's CPU-baseline leg may import it; the
product library never does.

The paper discretises the Gaussian prior field by a truncated KL expansion
theta(x) ~ m0(x) + sum_n m_n(x) theta_n with standard normal theta_n (Sec. 5,
Eq. truncKL). It does not say how the KL pairs are computed. The workloads here
use a separable exponential covariance
    C(x, x') = sigma^2 exp(-|x1-x1'|/lc) exp(-|x2-x2'|/lc),
whose eigenpairs are products of the analytic 1-D pairs of exp(-|s-t|/lc) on
[0,1] (the classical transcendental-equation solution, Ghanem & Spanos 1991).
Writing the interval as [-a, a] with a = 1/2 and c = 1/lc, x = omega*a:
  even modes: omega*tan(omega*a) = c,  phi = cos(omega(s-1/2)) / sqrt(a + sin(2 omega a)/(2 omega))
  odd  modes: omega + c*tan(omega*a) = 0, phi = sin(omega(s-1/2)) / sqrt(a - sin(2 omega a)/(2 omega))
  eigenvalue: lambda = 2c / (omega^2 + c^2)
1-D mode m has x in (m*pi/2, (m+1)*pi/2): even for m even, odd for m odd.
2-D pairs (m, n) carry sigma^2 lambda_m lambda_n and phi_m(x1) phi_n(x2); they
are ordered by eigenvalue descending, ties broken by smaller max(m, n) first,
then smaller m. The field value on a triangle is taken at its centroid (the
field is piecewise constant per element).
"""
import math

import numpy as np
from scipy.optimize import brentq


def _even_eq(x, a, c):
    # x = omega*a; cos-multiplied form of omega*tan(omega a) - c (no poles)
    return (x / a) * math.sin(x) - c * math.cos(x)


def _odd_eq(x, a, c):
    # cos-multiplied form of omega + c*tan(omega a)
    return (x / a) * math.cos(x) + c * math.sin(x)


def eig_1d(corr_len, n_modes):
    """1-D eigenpairs of exp(-|s-t|/corr_len) on [0,1], unit variance.

    Returns (lam, omega, parity) arrays of length n_modes, lam descending;
    parity 0 = even (cos) mode, 1 = odd (sin) mode.
    """
    a = 0.5
    c = 1.0 / corr_len
    lam = np.empty(n_modes)
    omega = np.empty(n_modes)
    parity = np.empty(n_modes, dtype=np.int64)
    for m in range(n_modes):
        lo = m * math.pi / 2.0
        hi = (m + 1) * math.pi / 2.0
        f = _even_eq if m % 2 == 0 else _odd_eq
        # the bracket endpoints are where the equation changes sign; pull
        # them in by a relative hair so no endpoint is an exact zero of sin/cos
        span = hi - lo
        x = brentq(f, lo + 1e-14 * span, hi - 1e-14 * span, args=(a, c),
                   xtol=1e-15, rtol=8.9e-16, maxiter=500)
        w = x / a
        omega[m] = w
        lam[m] = 2.0 * c / (w * w + c * c)
        parity[m] = m % 2
    return lam, omega, parity


def phi_1d(omega, parity, s):
    """Normalised 1-D eigenfunction evaluated at points s in [0,1]."""
    a = 0.5
    s = np.asarray(s, dtype=np.float64)
    if parity == 0:
        norm = math.sqrt(a + math.sin(2.0 * omega * a) / (2.0 * omega))
        return np.cos(omega * (s - 0.5)) / norm
    norm = math.sqrt(a - math.sin(2.0 * omega * a) / (2.0 * omega))
    return np.sin(omega * (s - 0.5)) / norm


def kl_pairs(corr_len, variance, K):
    """The K leading 2-D KL pairs: list of (lambda, m, n), lambda including variance."""
    lam1, _, _ = eig_1d(corr_len, K)
    pairs = []
    for m in range(K):
        for n in range(K):
            pairs.append((variance * (lam1[m] * lam1[n]), m, n))
    pairs.sort(key=lambda t: (-t[0], max(t[1], t[2]), t[1]))
    return pairs[:K]


def centroids(N):
    """Triangle centroids of the uniform N x N mesh, element order e = 2*(j*N+i) + t.

    t = 0: lower triangle (i,j),(i+1,j),(i+1,j+1); t = 1: upper (i,j),(i+1,j+1),(i,j+1).
    """
    h = 1.0 / N
    xc = np.empty(2 * N * N)
    yc = np.empty(2 * N * N)
    for j in range(N):
        for i in range(N):
            e = 2 * (j * N + i)
            xc[e] = (i + 2.0 / 3.0) * h
            yc[e] = (j + 1.0 / 3.0) * h
            xc[e + 1] = (i + 1.0 / 3.0) * h
            yc[e + 1] = (j + 2.0 / 3.0) * h
    return xc, yc


def kl_table(N, corr_len, variance, K):
    """Psi[k, e] = sqrt(lambda_k) phi_k(centroid_e), shape (K, 2N^2), FP64.

    The log-diffusion field of a particle theta is u = theta @ Psi (Eq. truncKL, m0 = 0).
    """
    lam1, om1, par1 = eig_1d(corr_len, K)
    xc, yc = centroids(N)
    psi = np.empty((K, xc.size))
    for k, (lam, m, n) in enumerate(kl_pairs(corr_len, variance, K)):
        psi[k] = math.sqrt(lam) * phi_1d(om1[m], par1[m], xc) * phi_1d(om1[n], par1[n], yc)
    return psi
