"""Forward response G_l(theta) and potential Phi_l(theta) on one mesh level (oracle).

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle; never imported by the
product library.

G = O o G_sol (Sec. 2.1): KL coefficients theta -> log-diffusion field
u = theta @ Psi (Eq. truncKL, m0 = 0, one value per triangle) -> kappa = exp(u)
(Sec. 5) -> P1 FEM solution p of -div(kappa grad p) = f, p = 0 on the boundary
-> observations p(d_n). The potential is Phi = 1/2 |Gamma^{-1/2}(y - G)|^2 with
Gamma = sigma^2 I (Eq. phi).
"""
import numpy as np

from . import fem
from . import kl
from . import matern


class Level:
    """One discretisation level: mesh N = 1/h, KL table and observation operator.

    cov: "sep_exp" (separable exponential, analytic KL) or "matern" (nu = 3/2, Nystrom KL);
    f: source term f(x, y), None for f = 1; bc: "dirichlet" (p = 0 on the boundary) or
    "flow_cell" (Example 5.3: p = 0 / 1 on x = 0 / 1, no flow on y = 0, 1, f = 0); m0: the prior
    mean of the field (Eq. truncKL)."""

    def __init__(self, N, corr_len, variance, K, obs_xy, f=None, cov="sep_exp", bc="dirichlet", m0=0.0):
        self.N = N
        if bc not in ("dirichlet", "flow_cell"):
            raise ValueError("bc must be 'dirichlet' or 'flow_cell'")
        self.bc = bc
        self.m0 = m0
        if cov == "sep_exp":
            self.psi = kl.kl_table(N, corr_len, variance, K)
        elif cov == "matern":
            self.psi = matern.kl_table(N, corr_len, variance, K)
        else:
            raise ValueError("cov must be 'sep_exp' or 'matern'")
        self.O = fem.observation_operator(N, obs_xy)
        self.f = f

    def field(self, theta):
        """u on every triangle for one particle (Eq. truncKL)."""
        return self.m0 + np.asarray(theta, dtype=np.float64) @ self.psi

    def solution(self, theta):
        if self.bc == "flow_cell":
            return fem.solve_flow_cell(self.N, np.exp(self.field(theta)))
        return fem.solve(self.N, np.exp(self.field(theta)), self.f)

    def G(self, theta):
        """Observation vector of one particle."""
        return self.O @ self.solution(theta)

    def G_batch(self, thetas):
        thetas = np.atleast_2d(thetas)
        return np.stack([self.G(t) for t in thetas])


def potential(G, y, sigma):
    """Phi = 1/2 sum_n ((y_n - G_n)/sigma)^2 for each row of G (Eq. phi, Gamma = sigma^2 I)."""
    G = np.atleast_2d(G)
    r = (np.asarray(y)[None, :] - G) / sigma
    return 0.5 * np.sum(r * r, axis=1)


class LinearLevel:
    """Linear-Gaussian stand-in for a level: G_l(theta) = A_l theta (test seam, no PDE)."""

    def __init__(self, A):
        self.A = np.asarray(A, dtype=np.float64)

    def G(self, theta):
        return self.A @ np.asarray(theta, dtype=np.float64)

    def G_batch(self, thetas):
        return np.atleast_2d(thetas) @ self.A.T
