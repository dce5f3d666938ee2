"""Pins of the oracle's SMC pieces: identities, monotonicity, resampling properties,
prior invariance of pCN, the Philox draw layout, closed-form linear-Gaussian
posteriors and evidence, and the exact cost identity of the update scheme."""
import math

import numpy as np
import pytest

from oracle import gaussian, philox, smc
from oracle.forward import potential


def test_kish_identity():
    w = np.random.default_rng(0).exponential(size=500)
    assert smc.ess(w) == pytest.approx(w.sum() ** 2 / np.sum(w * w), rel=1e-12)
    assert smc.cv(np.full(10, 3.0)) == 0.0


def test_cv_monotone_in_increment():
    """d/dDelta log(1 + cv^2) = 2 (E_Delta[a] - E_2Delta[a]) >= 0: cv never decreases along Delta."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = rng.gamma(2.0, 50.0, size=300)
        ds = np.linspace(0, 0.2, 200)
        c = np.array([smc.cv_of_increment(a, d) for d in ds])
        assert c[0] == 0.0
        assert np.all(np.diff(c) >= -1e-12)


def test_next_increment_hits_target_and_respects_bounds():
    rng = np.random.default_rng(2)
    a = rng.gamma(3.0, 40.0, size=1000)
    d = smc.next_increment(a, 1.0, 1.0, 1e-6)
    assert smc.cv_of_increment(a, d) == pytest.approx(1.0, abs=1e-10)
    # remaining step small enough: whole step taken
    assert smc.next_increment(a * 1e-6, 0.3, 1.0, 1e-6) == 0.3
    # equal potentials: cv == 0 for every step, whole step taken
    assert smc.next_increment(np.full(50, 7.0), 0.25, 1.0, 1e-6) == 0.25
    # target unreachable above eps: the minimum step eps is taken
    huge = np.concatenate([np.zeros(1), np.full(99, 1e12)])
    assert smc.next_increment(huge, 1.0, 1.0, 1e-6) == 1e-6


def test_log_mean_weight():
    a = np.random.default_rng(3).uniform(0, 50, 100)
    for d in (0.0, 0.01, 0.3):
        assert smc.log_mean_weight(a, d) == pytest.approx(math.log(np.mean(np.exp(-d * a))), rel=1e-12, abs=1e-14)
    # survives magnitudes where exp underflows without the shift
    big = a + 1e5
    assert smc.log_mean_weight(big, 1.0) == pytest.approx(smc.log_mean_weight(a, 1.0) - 1e5, rel=1e-12)


def test_systematic_resampling_properties():
    rng = np.random.default_rng(4)
    J = 257
    logw = rng.normal(0, 2, J)
    W = np.exp(logw - logw.max())
    W /= W.sum()
    for U in rng.uniform(0, 1, 50):
        anc = smc.systematic_resample(logw, U)
        assert anc.size == J and anc.min() >= 0 and anc.max() < J
        assert np.all(np.diff(anc) >= 0)
        cnt = np.bincount(anc, minlength=J)
        assert np.all(cnt >= np.floor(J * W) - 1e-9) and np.all(cnt <= np.ceil(J * W) + 1e-9)
    # offspring mean over U equals J * W (the scheme is unbiased)
    Us = (np.arange(4000) + 0.5) / 4000
    mean = np.mean([np.bincount(smc.systematic_resample(logw, U), minlength=J) for U in Us], axis=0)
    assert np.allclose(mean, J * W, atol=2e-3)
    # equal weights: identity
    assert np.array_equal(smc.systematic_resample(np.zeros(J), 0.5), np.arange(J))


def test_philox_uniform_and_normal_statistics():
    u = philox.uniforms_open(200000, 7, philox.PURPOSE_PCN_U, 12345)
    assert u.min() > 0 and u.max() <= 1
    hist = np.histogram(u, bins=20, range=(0, 1))[0]
    chi2 = np.sum((hist - 10000) ** 2 / 10000)
    assert chi2 < 45            # 19 dof, p ~ 0.001
    z = philox.normals(20000, 10, 3, philox.PURPOSE_PCN_XI, 99)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    c = np.corrcoef(z[:, :4].T)
    assert np.abs(c - np.eye(4)).max() < 0.03
    # distinct counters give distinct outputs; different seeds differ
    x = philox.philox4x32_10(np.arange(10000), 0, 0, 0, 1)[0]
    assert np.unique(x).size == 10000
    assert not np.array_equal(philox.normals(4, 4, 0, 2, 1), philox.normals(4, 4, 0, 2, 2))
    # odd K drops the last sine of each particle's final block
    assert np.array_equal(philox.normals(3, 5, 0, 2, 7), philox.normals(3, 6, 0, 2, 7)[:, :5])


def test_philox_known_answer_vectors():
    """Philox4x32-10 against the generator's published known-answer vectors (Salmon, Moraes, Dror
    and Shaw, SC 2011; the test vectors distributed with the authors' Random123 library, rounds = 10:
    counter words c0..c3, key words k0, k1, output words in the same order). A wrong multiplier,
    Weyl constant, round count or word order fails at least one of the three."""
    kat = [
        ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
         (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
        ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
         (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
        ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
         (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
    ]
    for ctr, (k0, k1), want in kat:
        got = philox.philox4x32_10(*ctr, k0 | (k1 << 32))
        assert tuple(int(w) for w in got) == want
    # the vectorised form gives the same words element by element
    c = np.array([kat[0][0][0], kat[1][0][0]], dtype=np.uint64)
    x0 = philox.philox4x32_10(c, c, c, c, 0)[0]
    assert int(x0[0]) == 0x6627e8d5


def test_pcn_preserves_prior_with_zero_potential():
    """Phi == 0: every proposal is accepted and N(0, I) is invariant under the pCN map."""
    K, J = 4, 20000
    s = smc.Sampler(lambda l, th: np.zeros(th.shape[0]), 1, K, J, n_mcmc=3, seed=5)
    s.step()
    assert s.done and s.path[-1]['accept'] == 1.0 and s.path[-1]['delta'] == 1.0
    m, v = s.moments()
    assert np.all(np.abs(m) < 4 / math.sqrt(J)) and np.all(np.abs(v - 1) < 0.05)


def _linear_problem(K=3, n=5, sigma=0.5, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.normal(0, 1, (n, K))
    y = A @ rng.normal(0, 1, K) + sigma * rng.normal(0, 1, n)
    return A, y, sigma


def test_single_level_smc_linear_gaussian():
    """Adaptive tempering + pCN reproduces the closed-form posterior and evidence."""
    A, y, sigma = _linear_problem()
    m_ex, C_ex = gaussian.posterior(A, y, sigma)
    lz_ex = gaussian.log_evidence(A, y, sigma)
    J = 4000
    ev = lambda l, th: potential(th @ A.T, y, sigma)
    s = smc.Sampler(ev, 1, 3, J, n_mcmc=10, s_pcn=0.5, seed=11).run()
    m, v = s.moments()
    se_m = np.sqrt(np.diag(C_ex) / J) * 3.0          # generous: SMC particles are correlated
    assert np.all(np.abs(m - m_ex) < 4 * se_m), (m, m_ex)
    assert np.allclose(v, np.diag(C_ex), rtol=0.15)
    assert s.log_z == pytest.approx(lz_ex, abs=0.15)
    assert all(p['kind'] == 'ITU' for p in s.path)
    assert s.beta == 1.0


def test_mls2mc_linear_gaussian_levels_and_cost_identity():
    """Two-level hierarchy A_l = A + 4^-l B: posterior on the fine level, path rules and the
    cost identity of Prop. Cost_Proposition (extended by n_mcmc steps and the J~ pre-evaluations)."""
    A, y, sigma = _linear_problem(K=3, n=6, sigma=0.2, seed=3)
    B = np.random.default_rng(9).normal(0, 1, A.shape)
    As = [A + 4.0 ** -(l + 1) * B * 8 for l in range(3)]
    J, nm, jt = 2000, 6, 100
    ev = lambda l, th: potential(th @ As[l].T, y, sigma)
    s = smc.Sampler(ev, 3, 3, J, J_tilde=jt, n_mcmc=nm, s_pcn=0.4, seed=21).run()
    m_ex, C_ex = gaussian.posterior(As[-1], y, sigma)
    m, v = s.moments()
    assert np.all(np.abs(m - m_ex) < 12 * np.sqrt(np.diag(C_ex) / J)), (m, m_ex)
    assert np.allclose(v, np.diag(C_ex), rtol=0.25)
    assert s.log_z == pytest.approx(gaussian.log_evidence(As[-1], y, sigma), abs=0.3)
    # path rules: first update is an ITU; an LU is followed by an ITU unless beta is already 1
    kinds = [(p['kind'], p['level']) for p in s.path]
    assert kinds[0] == ('ITU', 0)
    # cost identity
    expect = np.zeros(3, dtype=np.int64)
    expect[0] += J                                     # prior particles on level 1
    prev_level = 0
    for i, p in enumerate(s.path):
        if p['kind'] == 'ITU':
            expect[p['level']] += nm * J
            if 'cv_lu' in p:
                expect[p['level'] + 1] += jt           # discarded cv^LU pre-evaluations
        else:
            first_bridge = p['level'] != prev_level
            if first_bridge:
                expect[p['level']] += J                # new level on all particles (J~ reused)
            expect[p['level']] += nm * J
            expect[p['level'] - 1] += nm * J
        prev_level = p['level']
    assert np.array_equal(expect, s.evals), (expect, s.evals)
    assert s.level == 2 and s.beta == 1.0


def test_adaptive_maximum_level_scheme_stops_when_levels_agree():
    """Scheme u' (Sec. 4.5): at beta = 1 the level update is skipped, and the sampler stops, when
    cv^LU on the first J~ particles is below tau_min. Levels 2 and 3 of the hierarchy below differ
    by 1e-9 of the operator, so the run stops on level 2 and its posterior is that of level 2 (the
    closed form); with tau_min = 0 the same run goes on to level 3."""
    A, y, sigma = _linear_problem(K=3, n=6, sigma=0.2, seed=3)
    B = np.random.default_rng(9).normal(0, 1, A.shape)
    As = [A + 0.3 * B, A, A + 1e-9 * B]
    J, jt = 2000, 100
    ev = lambda l, th: potential(th @ As[l].T, y, sigma)
    s = smc.Sampler(ev, 3, 3, J, J_tilde=jt, n_mcmc=6, s_pcn=0.4, seed=21, tau_min=1e-3).run()
    assert s.done and s.terminated and s.level == 1 and s.beta == 1.0
    n_pre = 1 + sum(1 for p in s.path if p['level'] == 1 and 'cv_lu' in p)
    assert s.evals[2] == n_pre * jt                   # only J~ pre-evaluations on level 3
    m_ex, C_ex = gaussian.posterior(As[1], y, sigma)
    m, v = s.moments()
    assert np.all(np.abs(m - m_ex) < 12 * np.sqrt(np.diag(C_ex) / J))
    full = smc.Sampler(ev, 3, 3, J, J_tilde=jt, n_mcmc=6, s_pcn=0.4, seed=21).run()
    assert full.level == 2 and not full.terminated
    # both schemes take the same updates until beta first reaches 1 on level 2
    n = len(s.path)
    assert [(p['kind'], p['level']) for p in s.path] == [(p['kind'], p['level']) for p in full.path[:n]]


@pytest.mark.parametrize("proposal,s0", [("pcn", 0.05), ("rwm", 2.0)])
def test_adaptive_step_keeps_the_posterior_and_moves_toward_the_target_rate(proposal, s0):
    """With accept_target > 0 the step of each update is fixed before its moves (it depends on the
    finished updates only), so every update's kernel still leaves its target invariant: the
    linear-Gaussian posterior and evidence come out as in closed form, from a poor first step
    either way, each step follows the rule, and a step far off moves toward the target rate."""
    A, y, sigma = _linear_problem()
    m_ex, C_ex = gaussian.posterior(A, y, sigma)
    lz_ex = gaussian.log_evidence(A, y, sigma)
    J = 4000
    ev = lambda l, th: potential(th @ A.T, y, sigma)
    s = smc.Sampler(ev, 1, 3, J, n_mcmc=10, s_pcn=s0, seed=13, proposal=proposal, accept_target=0.3).run()
    m, v = s.moments()
    se_m = np.sqrt(np.diag(C_ex) / J) * 3.0
    assert np.all(np.abs(m - m_ex) < 4 * se_m), (m, m_ex)
    assert np.allclose(v, np.diag(C_ex), rtol=0.15)
    assert s.log_z == pytest.approx(lz_ex, abs=0.15)
    steps = [p['step'] for p in s.path]
    assert steps[0] == s0 and len(set(steps)) == len(steps)        # adapted between every update
    # each step follows the rule from the previous update's acceptance
    for a, b in zip(s.path[:-1], s.path[1:]):
        hi = 100.0 if proposal == "rwm" else 1.0
        assert b['step'] == min(hi, max(1e-4, a['step'] * math.exp(a['accept'] - 0.3)))
    # from a step far off, it moves in the direction that brings the rate toward the target
    assert (steps[-1] - steps[0]) * (s.path[0]['accept'] - 0.3) > 0


def test_distinct_ancestors_recorded():
    """n_unique of an update is the number of distinct ancestors its resampling kept: all J for a
    first update with equal potentials, fewer once the weights differ."""
    J = 500
    s = smc.Sampler(lambda l, th: np.zeros(th.shape[0]), 1, 2, J, n_mcmc=1, seed=3)
    s.step()
    assert s.path[-1]['n_unique'] == J
    A, y, sigma = _linear_problem()
    ev = lambda l, th: potential(th @ A.T, y, sigma)
    s = smc.Sampler(ev, 1, 3, J, n_mcmc=1, seed=3)
    s.step()
    U = philox.uniform_scalar(0, philox.PURPOSE_RESAMPLE, 3)
    phi0 = ev(0, philox.normals(J, 3, 0, philox.PURPOSE_PRIOR, 3))
    anc = smc.systematic_resample(-s.path[-1]['delta'] * phi0, U)
    assert s.path[-1]['n_unique'] == np.unique(anc).size < J


def test_population_chol_recovers_a_known_factor():
    """A population theta_j = mu + A z_j whose z_j are the 2K signed vectors +-sqrt(K) e_k (mean 0,
    covariance I exactly) has covariance A A^T, so with no ridge the factor is A itself (A lower
    triangular with a positive diagonal); the ridge adds ridge * (tr(C) / K + 1e-12) on the diagonal;
    a population of identical particles gets sqrt(ridge * 1e-12) I."""
    K = 5
    rng = np.random.default_rng(4)
    A = np.tril(rng.normal(0, 1, (K, K)))
    A[np.diag_indices(K)] = np.abs(A[np.diag_indices(K)]) + 0.5
    mu = rng.normal(0, 1, K)
    Z = np.concatenate([math.sqrt(K) * np.eye(K), -math.sqrt(K) * np.eye(K)])
    theta = np.tile(mu + Z @ A.T, (3, 1))             # J = 6K, every signed vector three times
    assert np.allclose(smc.population_chol(theta, ridge=0.0), A, rtol=0, atol=1e-12)
    L = smc.population_chol(theta, ridge=0.01)
    tr = np.sum(A * A) / K                            # tr(A A^T) / K
    assert np.allclose(L @ L.T, A @ A.T + 0.01 * (tr + 1e-12) * np.eye(K), rtol=0, atol=1e-12)
    assert np.allclose(np.triu(L, 1), 0.0)
    same = np.tile(mu, (7, 1))
    assert np.allclose(smc.population_chol(same, ridge=1e-4), 1e-8 * np.eye(K), rtol=0, atol=1e-14)


def test_rwm_cov_proposal_has_the_shaped_covariance():
    """theta' - theta = s L xi has covariance s^2 L L^T (a transposed factor would give s^2 L^T L)."""
    K, J = 4, 200000
    rng = np.random.default_rng(5)
    L = np.tril(rng.normal(0, 1, (K, K))) + 2 * np.eye(K)
    xi = philox.normals(J, K, 3, philox.PURPOSE_PCN_XI, 17)
    step = smc.rwm_cov_propose(np.zeros((J, K)), xi, 0.5, L)
    C = step.T @ step / J
    assert np.allclose(C, 0.25 * L @ L.T, atol=0.05 * np.abs(L @ L.T).max() * 0.25)
    assert not np.allclose(0.25 * L @ L.T, 0.25 * L.T @ L, atol=0.05 * np.abs(L @ L.T).max() * 0.25)


@pytest.mark.parametrize("accept_target", [0.0, 0.3])
def test_rwm_cov_keeps_the_posterior_and_accepts_more(accept_target):
    """The covariance-shaped random walk (covariance from the population before each update's moves)
    leaves every update's target invariant: the linear-Gaussian posterior and evidence in closed
    form; on this posterior, far narrower than the prior, it accepts more often than the plain
    random walk of the same step."""
    A, y, sigma = _linear_problem(sigma=0.1)
    m_ex, C_ex = gaussian.posterior(A, y, sigma)
    lz_ex = gaussian.log_evidence(A, y, sigma)
    J = 4000
    ev = lambda l, th: potential(th @ A.T, y, sigma)
    kw = dict(n_mcmc=5, s_pcn=2.38 / math.sqrt(3), seed=23, accept_target=accept_target)
    s = smc.Sampler(ev, 1, 3, J, proposal="rwm_cov", **kw).run()
    m, v = s.moments()
    se_m = np.sqrt(np.diag(C_ex) / J) * 3.0
    assert np.all(np.abs(m - m_ex) < 4 * se_m), (m, m_ex)
    assert np.allclose(v, np.diag(C_ex), rtol=0.15)
    assert s.log_z == pytest.approx(lz_ex, abs=0.15)
    plain = smc.Sampler(ev, 1, 3, J, proposal="rwm", **kw).run()
    acc = lambda smp: np.mean([p['accept'] for p in smp.path[len(smp.path) // 2:]])
    assert acc(s) > 2 * acc(plain), (acc(s), acc(plain))
