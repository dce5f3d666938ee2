"""GPU parity of the sampler steps (increment search, resampling, Philox draws, pCN) and of the
whole MLS^2MC / single-level SMC sampler against the FP64 oracle.

The oracle and the library use the same counter-based draw layout, so with one seed both consume
identical random numbers: on the FP64 path the whole update path (beta, zeta schedule, evidence,
particles) must agree to rounding, and statistically (3 Monte Carlo standard errors) against the
closed-form linear-Gaussian posterior.
"""
import numpy as np
import pytest

from oracle import gaussian, philox, smc
from oracle import forward as ofwd
from oracle.forward import potential
from paper_1709_09763_gb300 import native
from paper_1709_09763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _linear(K=3, n=5, sigma=0.5, seed=0, levels=1):
    rng = np.random.default_rng(seed)
    A = rng.normal(0, 1, (n, K))
    y = A @ rng.normal(0, 1, K) + sigma * rng.normal(0, 1, n)
    B = np.random.default_rng(seed + 100).normal(0, 1, A.shape)
    As = np.stack([A + 4.0 ** -(l + 1) * B * 8 for l in range(levels)]) if levels > 1 else A[None]
    return As, y, sigma


def _handle_linear(As, y, sigma, J, **kw):
    L, n, K = As.shape
    obs = np.full((n, 2), 0.5)
    return native.Handle(list(range(4, 4 + L)), K, obs, y, sigma, J=J, linear_A=As, **kw)


def test_philox_draws_match_oracle():
    As, y, s = _linear()
    h = _handle_linear(As, y, s, J=8, seed=0xDEADBEEF12345)
    for (J, K, ev, pu) in [(37, 5, 0, 1), (3, 16, 123456, 2), (1000, 1, 7, 3)]:
        g = h.philox_normals(J, K, ev, pu)
        o = philox.normals(J, K, ev, pu, 0xDEADBEEF12345)
        assert np.allclose(g, o, rtol=1e-14, atol=1e-15)
    u = h.philox_uniforms(513, 99, philox.PURPOSE_PCN_U)
    assert np.array_equal(u, philox.uniforms_open(513, 99, philox.PURPOSE_PCN_U, 0xDEADBEEF12345))


def test_next_increment_matches_oracle():
    As, y, s = _linear()
    h = _handle_linear(As, y, s, J=5000, tau_star=1.0, eps=1e-6)
    rng = np.random.default_rng(3)
    for n, dmax in [(5000, 1.0), (1000, 0.37), (33, 1.0), (1, 1.0)]:
        a = rng.gamma(2.0, 300.0, size=n)
        d, lm, c = h.next_increment(a, dmax)
        dref = smc.next_increment(a, dmax, 1.0, 1e-6)
        assert d == pytest.approx(dref, rel=1e-12), (n, dmax)
        assert lm == pytest.approx(smc.log_mean_weight(a, dref), rel=1e-12, abs=1e-13)
        assert c == pytest.approx(smc.cv_of_increment(a, dref), rel=1e-9, abs=1e-12)
    # the whole remaining step when cv stays below the target; equal potentials
    assert h.next_increment(rng.uniform(0, 1e-3, 100), 0.3)[0] == 0.3
    assert h.next_increment(np.full(64, 5.0), 0.25)[0] == 0.25
    # target unreachable above eps: eps is taken
    a = np.concatenate([np.zeros(1), np.full(99, 1e12)])
    assert h.next_increment(a, 1.0)[0] == 1e-6


def test_systematic_resampling():
    As, y, s = _linear()
    h = _handle_linear(As, y, s, J=4096)
    rng = np.random.default_rng(5)
    # dyadic weights: every partial sum is exact in any order, so indices match bit for bit
    for J in (4096, 1000, 7):
        w = 2.0 ** rng.integers(-12, 0, size=J)
        for U in (0.0, 0.5, 0.123456789, 0.999):
            ref = smc.systematic_resample(np.log(w), U)
            assert np.array_equal(h.systematic_resample(w, U), ref), (J, U)
    # general weights: offspring counts within {floor, ceil} of J W_j and nearly identical indices
    J = 4096
    w = np.exp(rng.normal(0, 3, J))
    W = w / w.sum()
    anc = h.systematic_resample(w, 0.37)
    cnt = np.bincount(anc, minlength=J)
    assert np.all(cnt >= np.floor(J * W) - 1e-9) and np.all(cnt <= np.ceil(J * W) + 1e-9)
    assert np.all(np.diff(anc) >= 0)
    assert np.mean(anc != smc.systematic_resample(np.log(w), 0.37)) < 1e-3


def _oracle_linear(As, y, sigma, J, **kw):
    ev = lambda l, th: potential(th @ As[l].T, y, sigma)
    return smc.Sampler(ev, As.shape[0], As.shape[2], J, **kw).run()


def _compare_paths(gp, op, tol):
    assert len(gp) == len(op)
    for g, o in zip(gp, op):
        assert g["kind"] == o["kind"]
        assert g["beta"] == pytest.approx(o["beta"], rel=tol, abs=tol)
        if g["kind"] == "LU":
            assert g["zeta"] == pytest.approx(o["zeta"], rel=tol, abs=tol)
        assert g["delta"] == pytest.approx(o["delta"], rel=tol, abs=tol)


def test_single_level_linear_gaussian_same_trajectory_and_closed_form():
    As, y, s = _linear()
    J = 4000
    kw = dict(n_mcmc=10, s_pcn=0.5, seed=11)
    h = _handle_linear(As, y, s, J=J, **kw)
    h.run()
    o = _oracle_linear(As, y, s, J, **kw)
    _compare_paths(h.path(), o.path, 1e-9)
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-8, atol=1e-9)
    m, v, lz = h.posterior_moments()
    assert lz == pytest.approx(o.log_z, rel=1e-10)
    m_ex, C_ex = gaussian.posterior(As[0], y, s)
    assert np.all(np.abs(m - m_ex) < 4 * 3 * np.sqrt(np.diag(C_ex) / J))
    assert np.allclose(v, np.diag(C_ex), rtol=0.15)
    assert lz == pytest.approx(gaussian.log_evidence(As[0], y, s), abs=0.15)


def test_mls2mc_linear_same_path_and_cost_identity():
    As, y, s = _linear(K=3, n=6, sigma=0.2, seed=3, levels=3)
    J = 2000
    kw = dict(J_tilde=100, n_mcmc=6, s_pcn=0.4, seed=21)
    h = _handle_linear(As, y, s, J=J, **kw)
    h.run()
    o = _oracle_linear(As, y, s, J, **kw)
    gp = h.path()
    _compare_paths(gp, o.path, 1e-9)
    assert any(p["kind"] == "LU" for p in gp) and gp[0]["kind"] == "ITU"
    st = h.state()
    assert st["evals"][:3] == list(o.evals)          # forward solves per level, exactly
    assert st["level"] == 2 and st["beta"] == 1.0
    assert st["log_z"] == pytest.approx(o.log_z, rel=1e-10)


def test_fem_fp64_sampler_matches_oracle_trajectory():
    """Two FEM levels h = 1/8, 1/16, K = 4, FP64 path: same update path and particles as the oracle."""
    K, J = 4, 300
    obs = wl.obs_grid(3)
    lv = [ofwd.Level(N, 0.3, 1.0, K, obs) for N in (8, 16)]
    th_true = np.random.default_rng(1).standard_normal(K)
    Gt = lv[1].G(th_true)
    sigma = 0.02 * np.abs(Gt).max()
    y = Gt + sigma * np.random.default_rng(2).standard_normal(obs.shape[0])
    kw = dict(J_tilde=50, n_mcmc=2, s_pcn=0.3, seed=5)
    h = native.Handle([8, 16], K, obs, y, sigma, corr_len=0.3, J=J, precision=native.SMC_FP64, rtol=1e-13, **kw)
    h.run()
    ev = lambda l, th: potential(lv[l].G_batch(th), y, sigma)
    o = smc.Sampler(ev, 2, K, J, **kw).run()
    _compare_paths(h.path(), o.path, 1e-7)
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-7, atol=1e-8)
    assert h.state()["evals"][:2] == list(o.evals)


def test_tempering_update_equals_first_itu_of_oracle():
    """smc_tempering_update from beta = 0 on level 0 is the scheme's first ITU: same particles."""
    As, y, s = _linear(K=4, n=6, sigma=0.3, seed=8)
    J = 1500
    kw = dict(n_mcmc=3, s_pcn=0.4, seed=77)
    h = _handle_linear(As, y, s, J=J, **kw)
    th0 = philox.normals(J, 4, 0, philox.PURPOSE_PRIOR, 77)
    h.set_particles(th0)
    info = h.tempering_update(0, 0.0, 3)
    ev = lambda l, th: potential(th @ As[l].T, y, s)
    o = smc.Sampler(ev, 1, 4, J, theta0=th0, **kw)
    o.step()
    th, phi = h.particles()
    assert info["beta"] == pytest.approx(o.beta, rel=1e-12)
    assert info["log_z_inc"] == pytest.approx(o.log_z, rel=1e-12)
    assert np.allclose(th, o.theta, rtol=1e-10, atol=1e-12)
    assert np.allclose(phi, o.phi, rtol=1e-10)
    assert h.state()["beta"] == 0.0          # the update-scheme state is untouched


@pytest.mark.parametrize("n", [8193, 20000, 100000])
def test_next_increment_many_particles_and_spreads(n):
    """The one-launch search with several particles per thread (n > 128 blocks x 64 threads) and
    potentials of very different spread (the increment then ranges over decades), against the
    oracle's bisection."""
    As, y, s = _linear()
    h = _handle_linear(As, y, s, J=n, tau_star=1.0, eps=1e-6)
    rng = np.random.default_rng(n)
    for a, dmax in [(rng.gamma(2.0, 3.0, n), 1.0), (rng.gamma(0.5, 3000.0, n), 1.0),
                    (rng.lognormal(3.0, 2.0, n), 0.01), (rng.normal(1e4, 1.0, n), 1.0)]:
        d, lm, c = h.next_increment(a, dmax)
        dref = smc.next_increment(a, dmax, 1.0, 1e-6)
        assert d == pytest.approx(dref, rel=1e-12), (n, dmax, d, dref)
        assert lm == pytest.approx(smc.log_mean_weight(a, dref), rel=1e-12, abs=1e-13)
        assert c == pytest.approx(smc.cv_of_increment(a, dref), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("J", [7, 40001])
def test_tempering_update_small_and_large_populations(J):
    """The one-launch resampling with one block (J = 7) and with several scan rounds per block and
    a ragged last block (J = 40001 over 128 blocks): same particles as the oracle's first ITU."""
    As, y, s = _linear(K=4, n=6, sigma=0.3, seed=8)
    kw = dict(n_mcmc=2, s_pcn=0.4, seed=91)
    h = _handle_linear(As, y, s, J=J, **kw)
    th0 = philox.normals(J, 4, 0, philox.PURPOSE_PRIOR, 91)
    h.set_particles(th0)
    info = h.tempering_update(0, 0.0, 2)
    ev = lambda l, th: potential(th @ As[l].T, y, s)
    o = smc.Sampler(ev, 1, 4, J, theta0=th0, **kw)
    o.step()
    th, phi = h.particles()
    assert info["beta"] == pytest.approx(o.beta, rel=1e-12)
    assert info["log_z_inc"] == pytest.approx(o.log_z, rel=1e-12, abs=1e-14)
    assert np.allclose(th, o.theta, rtol=1e-10, atol=1e-12)
    assert np.allclose(phi, o.phi, rtol=1e-10)


def test_adaptive_maximum_level_scheme_same_path_as_oracle():
    """Scheme u' (opts.tau_min > 0, Sec. 4.5): levels 2 and 3 differ by 1e-9 of the operator, so
    cv^LU at beta = 1 on level 2 is below tau_min and the run stops there: the same updates,
    evaluation counts (the J~ pre-evaluations on level 3 included) and particles as the oracle."""
    As0, y, s = _linear(K=3, n=6, sigma=0.2, seed=3)
    A = As0[0]
    B = np.random.default_rng(9).normal(0, 1, A.shape)
    As = np.stack([A + 0.3 * B, A, A + 1e-9 * B])
    J = 2000
    kw = dict(J_tilde=100, n_mcmc=6, s_pcn=0.4, seed=21)
    h = _handle_linear(As, y, s, J=J, tau_min=1e-3, **kw)
    h.run()
    o = smc.Sampler(lambda l, th: potential(th @ As[l].T, y, s), 3, 3, J, tau_min=1e-3, **kw).run()
    assert o.terminated and o.level == 1
    _compare_paths(h.path(), o.path, 1e-9)
    st = h.state()
    assert st["level"] == 1 and st["beta"] == 1.0
    assert st["evals"][:3] == list(o.evals)
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-8, atol=1e-9)
    info = h.step()
    assert info["status"] == 1 and h.state()["n_updates"] == st["n_updates"]


def test_increment_search_reports_numerical_singularity():
    """Degenerate weights (Sec. 4.3): when every potential is +inf no increment exists and the
    search reports SMC_ESINGULAR instead of a step."""
    As, y, s = _linear()
    h = _handle_linear(As, y, s, J=64)
    with pytest.raises(native.SmcError) as ei:
        h.next_increment(np.full(64, np.inf), 1.0)
    assert ei.value.code == native.SMC_ESINGULAR
    # the handle stays usable
    d, _, _ = h.next_increment(np.linspace(0.0, 1.0, 64), 1.0)
    assert d == 1.0


def test_bridging_update_equals_oracle_bridging_step():
    """smc_bridging_update (Sec. 4.1): Phi on both levels, the increment of zeta from zeta0 at the given
    beta, resampling with both potentials, pCN steps on the bridged target -- the oracle's bridging
    step with the same draws gives the same zeta, evidence factor, particles and potentials."""
    As, y, s = _linear(K=4, n=6, sigma=0.3, seed=9, levels=2)
    J, K = 1200, 4
    kw = dict(n_mcmc=3, s_pcn=0.4, seed=91)
    h = _handle_linear(As, y, s, J=J, **kw)
    th0 = philox.normals(J, K, 0, philox.PURPOSE_PRIOR, 91)
    h.set_particles(th0)
    beta, zeta0 = 0.7, 0.2
    info = h.bridging_update(0, beta, zeta0, 3)
    ev = lambda l, th: potential(th @ As[l].T, y, s)
    o = smc.Sampler(ev, 2, K, J, theta0=th0, **kw)
    phi_c, phi_f = o.evaluate(0, o.theta), o.evaluate(1, o.theta)
    delta, anc, cvw = o._reweight_resample(beta * (phi_f - phi_c), 1.0 - zeta0)
    o.theta, phi_c, phi_f = o.theta[anc], phi_c[anc], phi_f[anc]
    zeta = 1.0 if delta >= 1.0 - zeta0 else zeta0 + delta

    def target(prop):
        if prop is None:
            return beta * ((1.0 - zeta) * phi_c + zeta * phi_f), [phi_c, phi_f]
        pc, pf = o.evaluate(0, prop), o.evaluate(1, prop)
        return beta * ((1.0 - zeta) * pc + zeta * pf), [pc, pf]
    rate = o._mcmc(target)
    assert info["kind"] == "LU" and info["level"] == 1
    assert info["zeta"] == pytest.approx(zeta, rel=1e-12)
    assert info["delta"] == pytest.approx(delta, rel=1e-12)
    assert info["log_z_inc"] == pytest.approx(o.log_z, rel=1e-12)
    assert info["accept_rate"] == pytest.approx(rate, abs=1e-12)
    th, phi = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-10, atol=1e-12)
    assert np.allclose(phi, phi_c, rtol=1e-10)
    st = h.state()
    assert st["beta"] == 0.0 and st["level"] == 0       # the update-scheme state is untouched
    assert st["evals"][:2] == list(o.evals)               # both levels solved per proposal


def test_adaptive_step_and_distinct_ancestors_match_oracle():
    """Two FEM levels on the FP64 path with the adaptive Markov-kernel step (accept_target = 0.3):
    the same path, steps and distinct-ancestor counts per update as the oracle's sampler."""
    K, J = 4, 300
    obs = wl.obs_grid(3)
    lv = [ofwd.Level(N, 0.3, 1.0, K, obs) for N in (8, 16)]
    th_true = np.random.default_rng(3).standard_normal(K)
    Gt = lv[1].G(th_true)
    sigma = 0.02 * np.abs(Gt).max()
    y = Gt + sigma * np.random.default_rng(4).standard_normal(obs.shape[0])
    kw = dict(J_tilde=50, n_mcmc=2, s_pcn=0.6, seed=15, accept_target=0.3)
    h = native.Handle([8, 16], K, obs, y, sigma, corr_len=0.3, J=J, precision=native.SMC_FP64, rtol=1e-13, **kw)
    h.run()
    ev = lambda l, th: potential(lv[l].G_batch(th), y, sigma)
    o = smc.Sampler(ev, 2, K, J, **kw).run()
    gp = h.path()
    _compare_paths(gp, o.path, 1e-7)
    for g, r in zip(gp, o.path):
        assert g["n_unique"] == r["n_unique"]
        assert g["step"] == pytest.approx(r["step"], rel=1e-10)
    assert len({g["step"] for g in gp}) > 1
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("accept_target", [0.0, 0.3])
def test_covariance_shaped_walk_matches_oracle_linear(accept_target):
    """The covariance-shaped random walk (proposal "rwm_cov", not in the paper) on a three-level
    linear hierarchy, K = 4: the population covariance, its factor and the shaped steps on the GPU
    give the oracle's update path, steps, distinct-ancestor counts, particles and evidence."""
    As, y, s = _linear(K=4, n=6, sigma=0.1, seed=12, levels=3)
    J = 1500
    kw = dict(J_tilde=100, n_mcmc=3, s_pcn=2.38 / 2.0, seed=31, proposal="rwm_cov", accept_target=accept_target)
    h = _handle_linear(As, y, s, J=J, **kw)
    h.run()
    o = _oracle_linear(As, y, s, J, **kw)
    gp = h.path()
    _compare_paths(gp, o.path, 1e-9)
    for g, r in zip(gp, o.path):
        assert g["n_unique"] == r["n_unique"]
        assert g["accept_rate"] == pytest.approx(r["accept"], abs=1e-12)
        assert g["step"] == pytest.approx(r["step"], rel=1e-12)
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-9, atol=1e-10)
    assert h.posterior_moments()[2] == pytest.approx(o.log_z, rel=1e-10)
    assert h.state()["evals"][:3] == list(o.evals)


def test_covariance_shaped_walk_matches_oracle_fem():
    """Two FEM levels (1/8, 1/16) on the FP64 path with the covariance-shaped walk: the oracle's
    path and particles."""
    K, J = 4, 300
    obs = wl.obs_grid(3)
    lv = [ofwd.Level(N, 0.3, 1.0, K, obs) for N in (8, 16)]
    th_true = np.random.default_rng(7).standard_normal(K)
    Gt = lv[1].G(th_true)
    sigma = 0.02 * np.abs(Gt).max()
    y = Gt + sigma * np.random.default_rng(8).standard_normal(obs.shape[0])
    kw = dict(J_tilde=50, n_mcmc=2, s_pcn=1.0, seed=19, proposal="rwm_cov")
    h = native.Handle([8, 16], K, obs, y, sigma, corr_len=0.3, J=J, precision=native.SMC_FP64, rtol=1e-13, **kw)
    h.run()
    ev = lambda l, th: potential(lv[l].G_batch(th), y, sigma)
    o = smc.Sampler(ev, 2, K, J, **kw).run()
    _compare_paths(h.path(), o.path, 1e-7)
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-7, atol=1e-8)
    assert h.state()["evals"][:2] == list(o.evals)
