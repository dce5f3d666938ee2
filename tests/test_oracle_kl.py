"""Pins of the oracle's KL table against mathematics it does not itself use.

The 1-D pairs must satisfy their transcendental equations, the eigen-relation of
the covariance operator (checked by independent adaptive quadrature), the trace
identity sum(lambda) = variance, orthonormality (Gauss-Legendre quadrature), and a
Nystrom discretisation of the operator must reproduce the leading eigenvalues.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import kl


@pytest.mark.parametrize("lc", [0.05, 0.1, 0.3, 1.0])
def test_root_equations(lc):
    c = 1.0 / lc
    lam, om, par = kl.eig_1d(lc, 40)
    for w, p in zip(om, par):
        if p == 0:
            r = w * math.sin(w / 2) - c * math.cos(w / 2)
        else:
            r = w * math.cos(w / 2) + c * math.sin(w / 2)
        assert abs(r) < 1e-12 * max(w, c)
    assert np.all(np.diff(lam) < 0)
    assert np.all(np.diff(om) > 0)


@pytest.mark.parametrize("lc", [0.1, 0.3])
def test_eigen_relation_by_quadrature(lc):
    """integral_0^1 exp(-|s-t|/lc) phi(t) dt == lambda phi(s), quadrature split at the kink t = s."""
    lam, om, par = kl.eig_1d(lc, 8)
    for m in range(8):
        for s in (0.1, 0.37, 0.5, 0.93):
            f = lambda t: math.exp(-abs(s - t) / lc) * float(kl.phi_1d(om[m], par[m], t))
            v = quad(f, 0.0, s, epsabs=1e-14, epsrel=1e-13)[0] + quad(f, s, 1.0, epsabs=1e-14, epsrel=1e-13)[0]
            assert v == pytest.approx(lam[m] * float(kl.phi_1d(om[m], par[m], s)), abs=1e-11)


@pytest.mark.parametrize("lc", [0.1, 0.3])
def test_trace_identity(lc):
    """sum_m lambda_m = integral of C(s, s) = 1; the tail after M modes is below 2c/(pi^2 (M-1))."""
    M = 4000
    lam, _, _ = kl.eig_1d(lc, M)
    c = 1.0 / lc
    tail = 1.0 - lam.sum()
    assert 0.0 < tail < 2.0 * c / (math.pi ** 2 * (M - 1))


def test_orthonormality():
    x, wq = np.polynomial.legendre.leggauss(400)
    s = 0.5 * (x + 1.0)
    wq = 0.5 * wq
    lam, om, par = kl.eig_1d(0.1, 20)
    Phi = np.stack([kl.phi_1d(om[m], par[m], s) for m in range(20)])
    G = (Phi * wq) @ Phi.T
    assert np.abs(G - np.eye(20)).max() < 1e-12


def test_nystrom_eigenvalues():
    """Midpoint-rule Nystrom eigenvalues of the 1-D kernel converge to the analytic ones."""
    lc = 0.3
    n = 3000
    s = (np.arange(n) + 0.5) / n
    C = np.exp(-np.abs(s[:, None] - s[None, :]) / lc) / n
    ev = np.sort(np.linalg.eigvalsh(C))[::-1][:6]
    lam, _, _ = kl.eig_1d(lc, 6)
    assert np.allclose(ev, lam, rtol=2e-5)


def test_pairs_order_and_ties():
    pairs = kl.kl_pairs(0.3, 1.0, 32)
    lams = [p[0] for p in pairs]
    assert all(lams[i] >= lams[i + 1] for i in range(len(lams) - 1))
    assert (pairs[0][1], pairs[0][2]) == (0, 0)
    # symmetric pairs tie exactly; the smaller m comes first
    for a, b in zip(pairs, pairs[1:]):
        if a[0] == b[0]:
            assert max(a[1], a[2]) <= max(b[1], b[2])
            if max(a[1], a[2]) == max(b[1], b[2]):
                assert a[1] < b[1]
    assert (pairs[1][1], pairs[1][2]) == (0, 1) and (pairs[2][1], pairs[2][2]) == (1, 0)


def test_table_covariance_converges_to_kernel():
    """sum_k Psi[k,e] Psi[k,e'] approaches C(c_e, c_e') as K grows (separable exponential)."""
    N, lc = 8, 1.0
    xc, yc = kl.centroids(N)
    C = np.exp(-np.abs(xc[:, None] - xc[None, :]) / lc - np.abs(yc[:, None] - yc[None, :]) / lc)
    errs = []
    for K in (16, 64, 400):
        P = kl.kl_table(N, lc, 1.0, K)
        errs.append(np.abs(P.T @ P - C).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.06
    # truncation never overshoots the variance on the diagonal
    P = kl.kl_table(N, lc, 1.0, 64)
    assert np.all(np.sum(P * P, axis=0) <= 1.0 + 1e-12)
