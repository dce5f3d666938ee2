"""Truncated KL expansion of a Matern prior field by the Nystrom method (oracle).

TEST INFRASTRUCTURE ONLY: this module is part of the FP64 CPU oracle. Only the
tests, the smoke check and the benchmark's CPU-baseline leg may import it; the
product library never does.

Sec. 5 (Examples 5.1-5.3) uses a Matern prior covariance with smoothness nu = 3/2
in the parametrisation of Minasny & McBratney (2005), which the paper cites:
    C(r) = sigma^2 2^(1-nu)/Gamma(nu) z^nu K_nu(z),  z = 2 sqrt(nu) r / lc,
which for nu = 3/2 is sigma^2 (1 + z) exp(-z) with z = sqrt(6) r / lc. With
lc = 0.65 the ten leading KL terms carry 94.5 % of the variance, the figure the
paper gives for Example 5.1 (the r/lc and sqrt(3) r/lc conventions give 99.5 %
and 97.7 %).

The paper does not say how the KL pairs are computed. Reading used here: the
Nystrom method on the midpoint rule of an M x M cell grid (M = 32 by default,
weight w = 1/M^2): W C u = lambda u on the grid, then
    phi(x) = (1/lambda) sum_q w C(x, q) u(q)
extends u to any point, and Psi[k, e] = sqrt(lambda_k) phi_k(centroid_e).

Canonical basis. The grid is invariant under the reflections Sx: x -> 1-x,
Sy: y -> 1-y and the swap R: x <-> y, and C commutes with all three. Every
eigenvector is taken with a definite parity (sx, sy) under (Sx, Sy): the four
parity sectors are solved separately on the quarter grid (x, y < 1/2) with the
folded kernel
    A_s(p, q) = w [C(p, q) + sx C(p, Sx q) + sy C(p, Sy q) + sx sy C(p, Sx Sy q)],
which is symmetric. R maps sector (+, -) onto (-, +), so the two spectra are
equal and the eigenvalues of such pairs coincide; the (-, +) members are the
mirror images (x <-> y) of the (+, -) ones. Order: eigenvalue descending, where
eigenvalues within a relative 1e-9 count as equal and then the sector order
(+,+), (+,-), (-,+), (-,-) decides. Sign: every eigenvector of the sectors
(+,+), (+,-), (-,-) is signed so that sum_q w u(q) g(q) > 0 with the generic
weight g(x, y) = exp(0.7 x + 1.3 y); a (-, +) member inherits the sign of its
mirror partner.
"""
import math

import numpy as np

from .kl import centroids

SECTORS = ((1, 1), (1, -1), (-1, 1), (-1, -1))


def matern_cov(r, corr_len, variance, nu=1.5):
    """C(r) for nu = 1/2, 3/2 or 5/2 in the Minasny-McBratney parametrisation (closed forms)."""
    z = 2.0 * math.sqrt(nu) * np.asarray(r, dtype=np.float64) / corr_len
    if nu == 0.5:
        return variance * np.exp(-z)
    if nu == 1.5:
        return variance * (1.0 + z) * np.exp(-z)
    if nu == 2.5:
        return variance * (1.0 + z + z * z / 3.0) * np.exp(-z)
    raise ValueError("nu must be 1/2, 3/2 or 5/2")


def quarter_grid(M):
    """Cell centres with x, y < 1/2 of the M x M grid (M even), row-major in (ix, iy)."""
    c = (np.arange(M // 2) + 0.5) / M
    X, Y = np.meshgrid(c, c, indexing="ij")
    return X.ravel(), Y.ravel()


def _folded(px, py, qx, qy, sx, sy, corr_len, variance, nu):
    """sum over the four reflections of q of the parity-signed kernel values C(p, .)."""
    def c(ax, ay):
        return matern_cov(np.hypot(px[:, None] - ax[None, :], py[:, None] - ay[None, :]), corr_len, variance, nu)
    return c(qx, qy) + sx * c(1.0 - qx, qy) + sy * c(qx, 1.0 - qy) + sx * sy * c(1.0 - qx, 1.0 - qy)


def sector_matrix(M, sx, sy, corr_len, variance, nu=1.5):
    qx, qy = quarter_grid(M)
    return _folded(qx, qy, qx, qy, sx, sy, corr_len, variance, nu) / (M * M)


def _mirror(v, M):
    """u(x, y) -> u(y, x) on the quarter grid."""
    m = M // 2
    return v.reshape(m, m).T.ravel()


def kl_pairs(corr_len, variance, K, M=32, nu=1.5):
    """The K leading pairs: list of (lambda, sx, sy, u) with u on the quarter grid, sum_full w u^2 = 1."""
    qx, qy = quarter_grid(M)
    w = 1.0 / (M * M)
    g = np.exp(0.7 * qx + 1.3 * qy)
    found = []
    sols = {}
    for si, (sx, sy) in enumerate(SECTORS):
        if (sx, sy) == (-1, 1):
            continue
        lam, V = np.linalg.eigh(sector_matrix(M, sx, sy, corr_len, variance, nu))
        sols[(sx, sy)] = (lam[::-1], V[:, ::-1])
    for (sx, sy), (lam, V) in sols.items():
        for k in range(min(K, lam.size)):
            u = V[:, k] / math.sqrt(4.0 * w)              # full-grid normalisation sum w u^2 = 1
            # full-grid functional sum_q w u g over the four reflected copies of the quarter
            s = np.sum(w * u * (g + sx * np.exp(0.7 * (1 - qx) + 1.3 * qy) + sy * np.exp(0.7 * qx + 1.3 * (1 - qy))
                                + sx * sy * np.exp(0.7 * (1 - qx) + 1.3 * (1 - qy))))
            if s < 0:
                u = -u
            found.append((lam[k], SECTORS.index((sx, sy)), sx, sy, u))
            if (sx, sy) == (1, -1):
                found.append((lam[k], SECTORS.index((-1, 1)), -1, 1, _mirror(u, M)))
    # eigenvalue descending; within a relative 1e-9 the sector order decides
    found.sort(key=lambda t: -t[0])
    out = []
    i = 0
    while i < len(found):
        j = i
        while j + 1 < len(found) and found[i][0] - found[j + 1][0] <= 1e-9 * found[i][0]:
            j += 1
        out.extend(sorted(found[i:j + 1], key=lambda t: t[1]))
        i = j + 1
    return [(t[0], t[2], t[3], t[4]) for t in out[:K]]


def eigenfunction(pair, x, y, corr_len, variance, M=32, nu=1.5):
    """Nystrom extension phi(x) = (1/lambda) sum_q w C(x, q) u(q) at the points (x, y)."""
    lam, sx, sy, u = pair
    qx, qy = quarter_grid(M)
    out = np.empty(np.size(x))
    x = np.ravel(x)
    y = np.ravel(y)
    for a in range(0, x.size, 4096):
        b = min(x.size, a + 4096)
        out[a:b] = _folded(x[a:b], y[a:b], qx, qy, sx, sy, corr_len, variance, nu) @ u / (M * M)
    return out / lam


def kl_table(N, corr_len, variance, K, M=32, nu=1.5):
    """Psi[k, e] = sqrt(lambda_k) phi_k(centroid_e), shape (K, 2N^2), element order of kl.centroids."""
    xc, yc = centroids(N)
    psi = np.empty((K, xc.size))
    for k, pair in enumerate(kl_pairs(corr_len, variance, K, M, nu)):
        psi[k] = math.sqrt(pair[0]) * eigenfunction(pair, xc, yc, corr_len, variance, M, nu)
    return psi


def eigenvalues(corr_len, variance, K, M=32, nu=1.5):
    return np.array([p[0] for p in kl_pairs(corr_len, variance, K, M, nu)])
