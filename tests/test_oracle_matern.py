"""Pins of the oracle's Matern KL (Nystrom), the nine-source term and the random-walk kernel of
Sec. 5 against facts that do not come from the oracle's own code: the Bessel-function definition
of the Matern covariance, the variance fractions the paper states for Examples 5.1 and 5.3, brute
force on the full Nystrom matrix, the integral eigen-relation under an independent (finer)
quadrature, the symmetry group of the square, the mass of the sources, and the invariance of the
prior under a Metropolis kernel."""
import math

import numpy as np
import pytest
from scipy.special import gamma, kv
from scipy.stats import norm

from oracle import fem
from oracle import gaussian
from oracle import kl
from oracle import matern
from oracle import smc
from oracle.forward import potential


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_form_equals_bessel_definition(nu):
    """sigma^2 2^(1-nu)/Gamma(nu) z^nu K_nu(z), z = 2 sqrt(nu) r / lc (Minasny & McBratney 2005)."""
    r = np.linspace(1e-3, 2.0, 200)
    lc, var = 0.65, 1.7
    z = 2.0 * math.sqrt(nu) * r / lc
    ref = var * 2.0 ** (1 - nu) / gamma(nu) * z ** nu * kv(nu, z)
    assert np.allclose(matern.matern_cov(r, lc, var, nu), ref, rtol=1e-12, atol=0)
    assert matern.matern_cov(0.0, lc, var, nu) == var


def test_ten_terms_carry_the_variance_fraction_of_example_5_1():
    """Example 5.1: with lc = 0.65, nu = 3/2 and variance 1 the ten leading KL terms carry 94.5 %
    of the variance. The trace of the discrete operator is the variance exactly."""
    lam = []
    for sx, sy in matern.SECTORS:
        lam += list(np.linalg.eigvalsh(matern.sector_matrix(32, sx, sy, 0.65, 1.0)))
    lam = np.sort(lam)[::-1]
    assert abs(lam.sum() - 1.0) < 1e-12
    top = matern.eigenvalues(0.65, 1.0, 10)
    assert np.allclose(top, lam[:10], rtol=1e-12)
    assert 0.9445 < top.sum() < 0.9455


def _full_grid(M=32):
    c = (np.arange(M) + 0.5) / M
    X, Y = np.meshgrid(c, c, indexing="ij")
    return X.ravel(), Y.ravel()


def test_eigen_relation_under_a_finer_quadrature():
    """lambda phi(x) = integral C(x, y) phi(y) dy, the integral taken by the midpoint rule on a
    96 x 96 grid (not the 32 x 32 grid of the construction): agreement to the quadrature error."""
    lc, var = 0.65, 1.0
    pairs = matern.kl_pairs(lc, var, 10)
    rng = np.random.default_rng(4)
    px, py = rng.uniform(0, 1, 12), rng.uniform(0, 1, 12)
    Mf = 96
    fx, fy = _full_grid(Mf)
    C = matern.matern_cov(np.hypot(px[:, None] - fx[None, :], py[:, None] - fy[None, :]), lc, var)
    for pair in pairs:
        phi_f = matern.eigenfunction(pair, fx, fy, lc, var)
        lhs = pair[0] * matern.eigenfunction(pair, px, py, lc, var)
        rhs = C @ phi_f / (Mf * Mf)
        assert np.max(np.abs(lhs - rhs)) < 2e-3 * np.max(np.abs(phi_f))


def test_orthonormal_on_the_grid():
    """sum_q w phi_k(q) phi_l(q) = delta_kl on the full 32 x 32 grid (Nystrom values at the nodes)."""
    lc, var = 0.65, 1.0
    fx, fy = _full_grid()
    Phi = np.stack([matern.eigenfunction(p, fx, fy, lc, var) for p in matern.kl_pairs(lc, var, 16)])
    G = Phi @ Phi.T / (32 * 32)
    assert np.allclose(G, np.eye(16), atol=1e-11)


def test_reflection_parities_and_mirror_pairs():
    """phi(1-x, y) = sx phi(x, y), phi(x, 1-y) = sy phi(x, y); equal eigenvalues come in x <-> y
    mirror pairs, the (+,-) member first."""
    lc, var = 0.65, 1.0
    pairs = matern.kl_pairs(lc, var, 12)
    rng = np.random.default_rng(7)
    x, y = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50)
    for p in pairs:
        f = matern.eigenfunction(p, x, y, lc, var)
        assert np.allclose(matern.eigenfunction(p, 1 - x, y, lc, var), p[1] * f, atol=1e-12)
        assert np.allclose(matern.eigenfunction(p, x, 1 - y, lc, var), p[2] * f, atol=1e-12)
    for a, b in zip(pairs, pairs[1:]):
        if abs(a[0] - b[0]) <= 1e-9 * a[0]:
            assert (a[1], a[2], b[1], b[2]) == (1, -1, -1, 1)
            fa = matern.eigenfunction(a, x, y, lc, var)
            assert np.allclose(matern.eigenfunction(b, y, x, lc, var), fa, atol=1e-12)


def test_table_covariance_approaches_the_kernel():
    """sum_k Psi[k, e] Psi[k, e'] approaches C(c_e, c_e') as K grows (truncation error only)."""
    lc, var = 0.65, 1.0
    psi = matern.kl_table(8, lc, var, 120)
    xc, yc = kl.centroids(8)
    Cemp = psi.T @ psi
    C = matern.matern_cov(np.hypot(xc[:, None] - xc[None, :], yc[:, None] - yc[None, :]), lc, var)
    assert np.max(np.abs(Cemp - C)) < 0.03
    assert np.max(np.abs(matern.kl_table(8, lc, var, 10).T @ matern.kl_table(8, lc, var, 10) - C)) > 0.03


def test_nine_sources_mass_and_symmetry():
    """f(x, y) = g(x) g(y) with g the sum of the three 1-D Gaussian densities of Example 5.1
    (scipy's normal density here); each centre lies 0.25 or more inside the boundary, so f
    integrates to 9 up to the Gaussian tails (closed form with the normal CDF). The load vector
    carries that mass at fine h and inherits the mesh's symmetries (x <-> y and the half turn)."""
    sd = math.sqrt(0.001)
    g = lambda t: sum(norm.pdf(t, 0.25 * n, sd) for n in (1, 2, 3))
    rng = np.random.default_rng(2)
    for x, y in rng.uniform(0, 1, (20, 2)):
        assert fem.nine_sources(x, y) == pytest.approx(g(x) * g(y), rel=1e-12, abs=1e-300)
    mass_1d = sum(norm.cdf(1.0, 0.25 * n, sd) - norm.cdf(0.0, 0.25 * n, sd) for n in (1, 2, 3))
    assert mass_1d ** 2 == pytest.approx(9.0, rel=1e-12)
    N = 64
    b = fem.load_vector(N, fem.nine_sources)
    assert b.sum() == pytest.approx(9.0, rel=2e-3)
    B = b.reshape(N + 1, N + 1)
    assert np.allclose(B, B.T, atol=1e-12 * B.max())
    assert np.allclose(B, B[::-1, ::-1], atol=1e-12 * B.max())


def test_rwm_preserves_the_prior_with_zero_potential():
    """Phi == 0: the random walk is accepted with probability min(1, mu0(theta')/mu0(theta)) and
    N(0, I) stays invariant; the acceptance is below 1 (unlike pCN)."""
    K, J = 4, 20000
    step = 2.38 / math.sqrt(K)
    s = smc.Sampler(lambda l, th: np.zeros(th.shape[0]), 1, K, J, n_mcmc=5, s_pcn=step,
                    seed=5, proposal="rwm")
    s.step()
    # stationary acceptance E[min(1, exp(-(|theta + s xi|^2 - |theta|^2) / 2))], theta, xi ~ N(0, I)
    rng = np.random.default_rng(1)
    th, xi = rng.normal(size=(2, 2_000_000, K))
    acc = np.minimum(1.0, np.exp(-0.5 * (np.sum((th + step * xi) ** 2, 1) - np.sum(th * th, 1)))).mean()
    assert s.done and abs(s.path[-1]['accept'] - acc) < 0.01 and acc < 0.5
    m, v = s.moments()
    assert np.all(np.abs(m) < 5 / math.sqrt(J)) and np.all(np.abs(v - 1) < 0.06)


def test_rwm_single_level_smc_linear_gaussian():
    """Adaptive tempering with the random-walk kernel reproduces the closed-form posterior."""
    rng = np.random.default_rng(0)
    A = rng.normal(0, 1, (5, 3))
    y = A @ rng.normal(0, 1, 3) + 0.5 * rng.normal(0, 1, 5)
    m_ex, C_ex = gaussian.posterior(A, y, 0.5)
    J = 4000
    s = smc.Sampler(lambda l, th: potential(th @ A.T, y, 0.5), 1, 3, J, n_mcmc=10, s_pcn=0.6, seed=11,
                    proposal="rwm").run()
    m, v = s.moments()
    assert np.all(np.abs(m - m_ex) < 12 * np.sqrt(np.diag(C_ex) / J)), (m, m_ex)
    assert np.allclose(v, np.diag(C_ex), rtol=0.15)
    assert s.log_z == pytest.approx(gaussian.log_evidence(A, y, 0.5), abs=0.15)


def _expand(pair, M):
    """The quarter-grid vector of a pair on the full M x M grid, by its reflection parities."""
    _, sx, sy, u = pair
    m = M // 2
    q = u.reshape(m, m)
    full = np.empty((M, M))
    for ix in range(M):
        for iy in range(M):
            a, b, s = ix, iy, 1.0
            if a >= m:
                a, s = M - 1 - a, s * sx
            if b >= m:
                b, s = M - 1 - b, s * sy
            full[ix, iy] = s * q[a, b]
    return full.ravel()


def test_320_terms_carry_the_variance_fraction_of_example_5_3():
    """Example 5.3: with lc = 0.1, nu = 3/2 and variance 1 the 320 leading KL terms carry 95 % of
    the variance (64 x 64 Nystrom grid), and they are the 320 largest eigenvalues of the full
    4096 x 4096 Nystrom matrix, solved without the symmetry reduction (brute force)."""
    from scipy.linalg import eigh
    M, K = 64, 320
    assert matern.nystrom_cells(K) == M and matern.nystrom_cells(64) == 32
    top = matern.eigenvalues(0.1, 1.0, K)
    assert 0.945 < top.sum() < 0.955
    c = (np.arange(M) + 0.5) / M
    X, Y = np.meshgrid(c, c, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    W = matern.matern_cov(np.hypot(X[:, None] - X[None, :], Y[:, None] - Y[None, :]), 0.1, 1.0) / (M * M)
    assert abs(np.trace(W) - 1.0) < 1e-12
    lam = eigh(W, eigvals_only=True, subset_by_index=[M * M - K, M * M - 1])[::-1]
    assert np.allclose(top, lam, rtol=0, atol=1e-14)


def test_320_pairs_are_orthonormal_eigenpairs_of_the_full_nystrom_matrix():
    """W C u = lambda u and sum_q w u_k u_l = delta_kl on the full 64 x 64 grid for every one of
    the 320 pairs at lc = 0.1, each vector expanded from its quarter grid by its parities; the
    (+,+) and (-,-) vectors are even or odd under x <-> y, the (-,+) ones mirror a (+,-) one."""
    M, K = 64, 320
    pairs = matern.kl_pairs(0.1, 1.0, K)
    c = (np.arange(M) + 0.5) / M
    X, Y = np.meshgrid(c, c, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    W = matern.matern_cov(np.hypot(X[:, None] - X[None, :], Y[:, None] - Y[None, :]), 0.1, 1.0) / (M * M)
    U = np.stack([_expand(p, M) for p in pairs], axis=1)
    lam = np.array([p[0] for p in pairs])
    assert np.abs(W @ U - U * lam).max() < 1e-13
    assert np.allclose(U.T @ U / (M * M), np.eye(K), atol=1e-11)
    assert np.all(np.diff(lam) <= 1e-9 * lam[:-1])
    m = M // 2
    for p in pairs:
        q = p[3].reshape(m, m)
        if p[1] == p[2]:
            assert np.allclose(q.T, q, atol=1e-13) or np.allclose(q.T, -q, atol=1e-13)


def test_field_equals_the_table_contraction():
    """u = theta . Psi at every centroid, whether through the table or folded per sector."""
    th = np.random.default_rng(9).standard_normal(80)
    psi = matern.kl_table(8, 0.1, 1.0, 80)
    assert np.allclose(matern.field(8, th, 0.1, 1.0, 80), th @ psi, rtol=0, atol=1e-12)
    sub = np.array([0, 5, 77, 127])
    assert np.allclose(matern.kl_table_at(8, sub, 0.1, 1.0, 80), psi[:, sub], rtol=0, atol=1e-15)
