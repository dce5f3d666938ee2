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
and 97.7 %); with lc = 0.1 the 320 leading terms carry 95 %, the figure of
Example 5.3.

The paper does not say how the KL pairs are computed. Reading used here: the
Nystrom method on the midpoint rule of an M x M cell grid (weight w = 1/M^2):
W C u = lambda u on the grid, then
    phi(x) = (1/lambda) sum_q w C(x, q) u(q)
extends u to any point, and Psi[k, e] = sqrt(lambda_k) phi_k(centroid_e).
M = 32 for up to 64 terms and M = 64 beyond (nystrom_cells): at lc = 0.1 the
sum of the 320 leading eigenvalues moves by 2.2e-4 between M = 64 and M = 96.

Canonical basis. The grid is invariant under the reflections Sx: x -> 1-x,
Sy: y -> 1-y and the swap R: x <-> y, and C commutes with all three. Every
eigenvector is taken with a definite parity (sx, sy) under (Sx, Sy): the four
parity sectors are solved separately on the quarter grid (x, y < 1/2) with the
folded kernel
    A_s(p, q) = w [C(p, q) + sx C(p, Sx q) + sy C(p, Sy q) + sx sy C(p, Sx Sy q)],
which is symmetric. R maps sector (+, -) onto (-, +), so the two spectra are
equal and the eigenvalues of such pairs coincide; the (-, +) members are the
mirror images (x <-> y) of the (+, -) ones. R maps the sectors (+, +) and
(-, -) onto themselves; each is split further into the vectors even and odd
under R (u(y, x) = +-u(x, y)), solved on the orthonormal basis of such vectors.
Without that split, R-even and R-odd eigenvalues that lie within a relative
1e-8 of each other (there are such pairs among the 320 leading ones at
lc = 0.1) would leave the eigenvectors of a sector mixtures that depend on
rounding. Order: eigenvalue descending, where eigenvalues within a relative
1e-9 count as equal and then the sector order (+,+), (+,-), (-,+), (-,-)
decides (R-even before R-odd). Sign: every eigenvector of the sectors (+,+),
(+,-), (-,-) is signed so that sum_q w u(q) g(q) > 0 with the generic weight
g(x, y) = exp(0.7 x + 1.3 y); a (-, +) member inherits the sign of its mirror
partner.
"""
import math

import numpy as np

from .kl import centroids

SECTORS = ((1, 1), (1, -1), (-1, 1), (-1, -1))


def nystrom_cells(K):
    """Cells per side of the Nystrom grid for K terms (the reading above)."""
    return 32 if K <= 64 else 64


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


def _cells_of(u):
    return 2 * math.isqrt(np.size(u))


def _folded(px, py, qx, qy, sx, sy, corr_len, variance, nu):
    """sum over the four reflections of q of the parity-signed kernel values C(p, .)."""
    def c(ax, ay):
        return matern_cov(np.hypot(px[:, None] - ax[None, :], py[:, None] - ay[None, :]), corr_len, variance, nu)
    return c(qx, qy) + sx * c(1.0 - qx, qy) + sy * c(qx, 1.0 - qy) + sx * sy * c(1.0 - qx, 1.0 - qy)


def sector_matrix(M, sx, sy, corr_len, variance, nu=1.5):
    qx, qy = quarter_grid(M)
    return _folded(qx, qy, qx, qy, sx, sy, corr_len, variance, nu) / (M * M)


def swap_basis(M, parity):
    """Orthonormal basis (columns) of the quarter-grid vectors with u(iy, ix) = parity u(ix, iy):
    e_(i,i) for the diagonal (parity +1 only) and (e_(i,j) + parity e_(j,i)) / sqrt(2), i < j."""
    m = M // 2
    cols = []
    for ix in range(m):
        for iy in range(ix, m):
            v = np.zeros(m * m)
            if ix == iy:
                if parity < 0:
                    continue
                v[ix * m + iy] = 1.0
            else:
                v[ix * m + iy] = 1.0 / math.sqrt(2.0)
                v[iy * m + ix] = parity / math.sqrt(2.0)
            cols.append(v)
    return np.array(cols).T


def _mirror(v, M):
    """u(x, y) -> u(y, x) on the quarter grid."""
    m = M // 2
    return v.reshape(m, m).T.ravel()


# solved sub-problems: (sector index, sx, sy, swap parity or 0 for none); (-, +) comes from (+, -)
_SUBSECTORS = ((0, 1, 1, 1), (0, 1, 1, -1), (1, 1, -1, 0), (3, -1, -1, 1), (3, -1, -1, -1))


def kl_pairs(corr_len, variance, K, M=None, nu=1.5):
    """The K leading pairs: list of (lambda, sx, sy, u) with u on the quarter grid, sum_full w u^2 = 1."""
    M = M or nystrom_cells(K)
    qx, qy = quarter_grid(M)
    w = 1.0 / (M * M)
    # the generic weight summed over the four reflected copies of the quarter grid, per sector
    e = lambda ax, ay: np.exp(0.7 * ax + 1.3 * ay)
    found = []
    for sec, sx, sy, par in _SUBSECTORS:
        A = sector_matrix(M, sx, sy, corr_len, variance, nu)
        if par:
            B = swap_basis(M, par)
            lam, V = np.linalg.eigh(B.T @ A @ B)
            V = B @ V
        else:
            lam, V = np.linalg.eigh(A)
        lam, V = lam[::-1], V[:, ::-1]
        gs = e(qx, qy) + sx * e(1 - qx, qy) + sy * e(qx, 1 - qy) + sx * sy * e(1 - qx, 1 - qy)
        for k in range(min(K, lam.size)):
            u = V[:, k] / math.sqrt(4.0 * w)              # full-grid normalisation sum w u^2 = 1
            if np.sum(w * u * gs) < 0:
                u = -u
            found.append((lam[k], sec, -par, sx, sy, u))
            if sec == 1:
                found.append((lam[k], 2, 0, -1, 1, _mirror(u, M)))
    # eigenvalue descending; within a relative 1e-9 the sector order (R-even first) decides
    found.sort(key=lambda t: -t[0])
    out = []
    i = 0
    while i < len(found):
        j = i
        while j + 1 < len(found) and found[i][0] - found[j + 1][0] <= 1e-9 * found[i][0]:
            j += 1
        out.extend(sorted(found[i:j + 1], key=lambda t: (t[1], t[2])))
        i = j + 1
    return [(t[0], t[3], t[4], t[5]) for t in out[:K]]


def eigenfunction(pair, x, y, corr_len, variance, nu=1.5):
    """Nystrom extension phi(x) = (1/lambda) sum_q w C(x, q) u(q) at the points (x, y)."""
    lam, sx, sy, u = pair
    M = _cells_of(u)
    qx, qy = quarter_grid(M)
    out = np.empty(np.size(x))
    x = np.ravel(x)
    y = np.ravel(y)
    for a in range(0, x.size, 4096):
        b = min(x.size, a + 4096)
        out[a:b] = _folded(x[a:b], y[a:b], qx, qy, sx, sy, corr_len, variance, nu) @ u / (M * M)
    return out / lam


def _extend(pairs, x, y, coef, corr_len, variance, nu):
    """sum over pairs of coef[k, :] times the Nystrom sums sum_q w C(x, q) u_k(q), per point:
    returns (rows of coef) x (points). Per chunk of points the kernel is evaluated once at q and
    its three mirror images, folded per sector and applied to all pairs of that sector."""
    M = _cells_of(pairs[0][3])
    qx, qy = quarter_grid(M)
    x, y = np.ravel(x), np.ravel(y)
    by_sector = {s: [k for k, p in enumerate(pairs) if (p[1], p[2]) == s] for s in SECTORS}
    out = np.zeros((coef.shape[0], x.size))
    for a in range(0, x.size, 2048):
        b = min(x.size, a + 2048)
        px, py = x[a:b, None], y[a:b, None]
        c = [matern_cov(np.hypot(px - ax[None, :], py - ay[None, :]), corr_len, variance, nu)
             for ax, ay in ((qx, qy), (1.0 - qx, qy), (qx, 1.0 - qy), (1.0 - qx, 1.0 - qy))]
        for (sx, sy), ks in by_sector.items():
            if not ks:
                continue
            F = (c[0] + sx * c[1] + sy * c[2] + sx * sy * c[3]) / (M * M)
            U = np.stack([pairs[k][3] for k in ks], axis=1)        # Q x (pairs of the sector)
            out[:, a:b] += coef[:, ks] @ (F @ U).T
    return out


def kl_table_at(N, elems, corr_len, variance, K, M=None, nu=1.5):
    """Psi[k, e] for the element indices elems (element order of kl.centroids): shape (K, len)."""
    pairs = kl_pairs(corr_len, variance, K, M, nu)
    xc, yc = centroids(N)
    elems = np.asarray(elems)
    coef = np.diag([1.0 / math.sqrt(p[0]) for p in pairs])          # sqrt(lambda) / lambda
    return _extend(pairs, xc[elems], yc[elems], coef, corr_len, variance, nu)


def kl_table(N, corr_len, variance, K, M=None, nu=1.5):
    """Psi[k, e] = sqrt(lambda_k) phi_k(centroid_e), shape (K, 2N^2), element order of kl.centroids."""
    return kl_table_at(N, np.arange(2 * N * N), corr_len, variance, K, M, nu)


def field(N, theta, corr_len, variance, K, M=None, nu=1.5):
    """u(centroid_e) = sum_k theta_k Psi[k, e] for one parameter vector, without the full table."""
    pairs = kl_pairs(corr_len, variance, K, M, nu)
    xc, yc = centroids(N)
    coef = (np.asarray(theta, dtype=np.float64) / np.sqrt([p[0] for p in pairs]))[None, :]
    return _extend(pairs, xc, yc, coef, corr_len, variance, nu)[0]


def eigenvalues(corr_len, variance, K, M=None, nu=1.5):
    return np.array([p[0] for p in kl_pairs(corr_len, variance, K, M, nu)])
