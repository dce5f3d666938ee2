"""Example 5.3 at the paper's size on the GPU path against the FP64 oracle: the 320-term Matern KL
(64 x 64 Nystrom grid) on 1/16 .. 1/256, the synthesis of 320 terms (five tensor-core
contractions of 64 terms each, their partial fields summed in FP64), G parity of the flow cell on
every level, and a short MLS^2MC run under the scheme u' with the random-walk kernel."""
import json
import math
import os

import numpy as np
import pytest

from oracle import fem as ofem
from oracle import forward as ofwd
from oracle import matern as omat
from oracle import smc
from oracle.forward import potential
from paper_1709_09763_gb300 import native
from paper_1709_09763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
W = wl.WORKLOADS["example_5_3_full"]


@pytest.fixture(scope="module")
def setup():
    from paper_1709_09763_gb300 import build
    build.build()
    with open(os.path.join(GOLD, f"data_{W.name}.json")) as f:
        d = json.load(f)
    obs = wl.obs_grid(W.obs_per_side)
    h = native.Handle(list(W.inv_h), W.K, obs, d["y"], d["sigma"], corr_len=W.corr_len,
                      precision=native.SMC_MIXED, cov="matern", bc="flow_cell")
    yield h, d, obs
    h.close()


def _rel(a, b):
    return np.max(np.abs(a - b), axis=-1) / np.max(np.abs(b), axis=-1)


def test_320_term_tables_match_oracle(setup):
    h, _, _ = setup
    lam_ref = omat.eigenvalues(W.corr_len, 1.0, W.K)
    for l, N in enumerate(W.inv_h):
        psi, lam = h.kl_table(l, N)
        assert np.allclose(lam, lam_ref, rtol=0, atol=1e-15)
        el = np.arange(2 * N * N) if N <= 32 else np.random.default_rng(N).choice(2 * N * N, 200, replace=False)
        assert np.abs(psi[:, el] - omat.kl_table_at(N, el, W.corr_len, 1.0, W.K)).max() < 1e-12, N


def test_example_5_3_full_likelihood_parity(setup):
    """1e-6 of the oracle on 1/16 .. 1/128 (four particles) and on 1/256 (one particle, its field
    from the oracle's per-sector extension); p = x for theta = 0 and the maximum principle."""
    h, d, obs = setup
    y, sigma = np.array(d["y"]), d["sigma"]
    theta = wl.particles(4, W.K, 541)
    for l, N in enumerate(W.inv_h):
        G0, _ = h.eval_likelihood(l, np.zeros((1, W.K)))
        assert np.max(np.abs(G0 - obs[:, 0][None, :])) < 1e-6, N
        if N <= 128:
            Gr = ofwd.Level(N, W.corr_len, 1.0, W.K, obs, cov="matern", bc="flow_cell").G_batch(theta)
            th = theta
        else:
            th = theta[:1]
            u = omat.field(N, th[0], W.corr_len, 1.0, W.K)
            Gr = (ofem.observation_operator(N, obs) @ ofem.solve_flow_cell(N, np.exp(u)))[None, :]
        G, Phi = h.eval_likelihood(l, th)
        assert _rel(G, Gr).max() < 1e-6, N
        assert np.allclose(Phi, potential(Gr, y, sigma), rtol=1e-4)
        assert np.all((G > -1e-9) & (G < 1 + 1e-9))


def test_example_5_3_full_mls2mc_run(setup):
    """MLS^2MC on 1/16 .. 1/256 with J = 250 (the paper's smallest), one random-walk step per update
    (covariance 2.38^2 / 320), scheme u' (tau_min = 0.001): reaches beta = 1 on some level, every
    update path entry well formed, finite posterior moments of the 320 coefficients."""
    _, d, obs = setup
    h = native.Handle(list(W.inv_h), W.K, obs, d["y"], d["sigma"], corr_len=W.corr_len, J=250, n_mcmc=1,
                      s_pcn=2.38 / math.sqrt(W.K), precision=native.SMC_MIXED, seed=W.seed_sampler, cov="matern",
                      bc="flow_cell", proposal="rwm", tau_min=W.tau_min)
    h.run()
    st = h.state()
    assert st["beta"] == 1.0 and 0 <= st["level"] < len(W.inv_h)
    path = h.path()
    assert path and all(0.0 <= p["accept_rate"] <= 1.0 for p in path)
    mean, var, log_z = h.posterior_moments()
    assert mean.shape == (W.K,) and np.all(np.isfinite(mean)) and np.all(var > 0) and np.isfinite(log_z)
    h.close()


def test_320_term_mls2mc_path_equals_oracle_sampler(setup):
    """The 320-term flow cell on the levels 1/16, 1/32, 1/64 with J = 100, one random-walk step per
    update, scheme u' (Sec. 4.5): the mixed-precision sampler takes the oracle sampler's update path
    (kinds, beta, zeta, increments within the mixed path's 1e-6 potential error), the same evaluation
    counts per level, and the same particles (the draws are shared, so equal accept decisions give
    equal rows)."""
    _, d, obs = setup
    y, sigma = np.array(d["y"]), d["sigma"]
    levels = (16, 32, 64)
    J = 100
    kw = dict(J_tilde=32, n_mcmc=1, s_pcn=2.38 / math.sqrt(W.K), seed=W.seed_sampler)
    h = native.Handle(list(levels), W.K, obs, y, sigma, corr_len=W.corr_len, J=J, precision=native.SMC_MIXED,
                      cov="matern", bc="flow_cell", proposal="rwm", tau_min=W.tau_min, **kw)
    h.run()
    lv = [ofwd.Level(N, W.corr_len, 1.0, W.K, obs, cov="matern", bc="flow_cell") for N in levels]
    o = smc.Sampler(lambda l, th: potential(lv[l].G_batch(th), y, sigma), len(levels), W.K, J, proposal="rwm",
                    tau_min=W.tau_min, **kw).run()
    gp = h.path()
    assert len(gp) == len(o.path) and len(gp) >= 6
    assert any(r["kind"] == "LU" for r in o.path)
    for g, r in zip(gp, o.path):
        assert g["kind"] == r["kind"]
        assert g["beta"] == pytest.approx(r["beta"], rel=1e-4, abs=1e-6)
        assert g["delta"] == pytest.approx(r["delta"], rel=1e-4, abs=1e-6)
        if r["kind"] == "LU":
            assert g["zeta"] == pytest.approx(r["zeta"], rel=1e-4, abs=1e-6)
    st = h.state()
    assert st["evals"][:3] == list(o.evals)
    assert st["level"] == o.level and st["beta"] == 1.0
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-9, atol=1e-9)
    assert h.posterior_moments()[2] == pytest.approx(o.log_z, rel=1e-5)
    h.close()
