"""Closed-form posterior and evidence of a linear-Gaussian inverse problem (oracle reference).

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle; never imported by the
product library.

With G(theta) = A theta, prior N(0, I) and noise N(0, sigma^2 I), the posterior
of Eq. BayesBIP is Gaussian with covariance C = (I + A^T A / sigma^2)^{-1} and
mean m = C A^T y / sigma^2. With the potential of Eq. phi (no likelihood
normalising constant) the evidence of Eq. evidence is
Z = det(I + A^T A / sigma^2)^{-1/2} exp(-1/2 y^T (sigma^2 I + A A^T)^{-1} y).
A tempered target exp(-beta Phi) mu0 is the same problem with sigma^2 / beta.
"""
import numpy as np


def posterior(A, y, sigma, beta=1.0):
    A = np.asarray(A, dtype=np.float64)
    K = A.shape[1]
    P = np.eye(K) + beta * (A.T @ A) / sigma ** 2
    C = np.linalg.inv(P)
    m = C @ (beta * A.T @ np.asarray(y)) / sigma ** 2
    return m, C


def log_evidence(A, y, sigma):
    A = np.asarray(A, dtype=np.float64)
    n, K = A.shape
    _, logdet = np.linalg.slogdet(np.eye(K) + (A.T @ A) / sigma ** 2)
    S = sigma ** 2 * np.eye(n) + A @ A.T
    y = np.asarray(y, dtype=np.float64)
    return -0.5 * logdet - 0.5 * y @ np.linalg.solve(S, y)
