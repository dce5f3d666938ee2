"""The flow cell of Example 5.3 on the GPU path (p = 0 / 1 on x = 0 / 1, no flow on y = 0, 1,
f = 0, Matern prior) against the FP64 oracle: the constant-field solution, G parity on every
level, and the sampler's path under the scheme u' with the random-walk kernel on the FP64 path."""
import math

import numpy as np
import pytest

from oracle import forward as ofwd
from oracle import smc
from oracle.forward import potential
from paper_1709_09763_gb300 import native
from paper_1709_09763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
K, LC = 32, 0.1


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _rel(a, b):
    return np.max(np.abs(a - b), axis=-1) / np.max(np.abs(b), axis=-1)


@pytest.mark.parametrize("prec", [native.SMC_MIXED, native.SMC_FP64])
def test_flow_cell_constant_field_gives_the_linear_pressure(prec):
    """theta = 0 (kappa = 1): p(x, y) = x at every node, so G is the observations' x coordinates."""
    obs = wl.obs_grid(7)
    levels = [8, 16, 32, 64] if prec == native.SMC_MIXED else [8, 16, 32]
    h = native.Handle(levels, K, obs, np.zeros(49), 0.045, corr_len=LC, precision=prec, cov="matern",
                      bc="flow_cell")
    tol = 1e-6 if prec == native.SMC_MIXED else 1e-12
    for l in range(len(levels)):
        G, _ = h.eval_likelihood(l, np.zeros((2, K)))
        assert np.max(np.abs(G - obs[:, 0][None, :])) < tol, levels[l]


@pytest.mark.parametrize("N,n", [(128, 4), (256, 2)])
def test_flow_cell_large_levels(N, n):
    """1/128 and 1/256 (fine levels in device memory): parity with the oracle and p = x for
    kappa = 1."""
    obs = wl.obs_grid(7)
    y = np.full(49, 0.5)
    h = native.Handle([N], K, obs, y, 0.045, corr_len=LC, precision=native.SMC_MIXED, cov="matern",
                      bc="flow_cell")
    G0, _ = h.eval_likelihood(0, np.zeros((1, K)))
    assert np.max(np.abs(G0 - obs[:, 0][None, :])) < 1e-6
    theta = wl.particles(n, K, 534)
    G, Phi = h.eval_likelihood(0, theta)
    Gr = ofwd.Level(N, LC, 1.0, K, obs, cov="matern", bc="flow_cell").G_batch(theta)
    assert _rel(G, Gr).max() < 1e-6


@pytest.mark.parametrize("prec", [native.SMC_MIXED, native.SMC_FP64])
def test_flow_cell_likelihood_parity(prec):
    obs = wl.obs_grid(7)
    levels = [8, 16, 32, 64] if prec == native.SMC_MIXED else [8, 16, 32]
    tol = 1e-6 if prec == native.SMC_MIXED else 1e-10
    y = np.full(49, 0.5)
    h = native.Handle(levels, K, obs, y, 0.045, corr_len=LC, precision=prec, cov="matern", bc="flow_cell")
    theta = wl.particles(6, K, 533)
    for l, N in enumerate(levels):
        lv = ofwd.Level(N, LC, 1.0, K, obs, cov="matern", bc="flow_cell")
        Gr = lv.G_batch(theta)
        G, Phi = h.eval_likelihood(l, theta)
        assert _rel(G, Gr).max() < tol, N
        assert np.allclose(Phi, potential(Gr, y, 0.045), rtol=100 * tol)
        assert np.all((G > -1e-9) & (G < 1 + 1e-9))          # maximum principle


def test_flow_cell_sampler_path_under_u_prime():
    """FP64 path, levels 1/8 and 1/16, one random-walk step per update, scheme u' (tau_min > 0):
    the same update path, evaluation counts and particles as the oracle."""
    obs = wl.obs_grid(7)
    lv = [ofwd.Level(N, LC, 1.0, K, obs, cov="matern", bc="flow_cell") for N in (8, 16)]
    th_true = np.random.default_rng(61).standard_normal(K)
    y = lv[1].G(th_true) + 0.045 * np.random.default_rng(62).standard_normal(49)
    J = 300
    kw = dict(J_tilde=50, n_mcmc=1, s_pcn=2.38 / math.sqrt(K), seed=63)
    h = native.Handle([8, 16], K, obs, y, 0.045, corr_len=LC, J=J, precision=native.SMC_FP64, rtol=1e-13,
                      cov="matern", bc="flow_cell", proposal="rwm", tau_min=1e-3, **kw)
    h.run()
    o = smc.Sampler(lambda l, th: potential(lv[l].G_batch(th), y, 0.045), 2, K, J, proposal="rwm", tau_min=1e-3,
                    **kw).run()
    gp = h.path()
    assert len(gp) == len(o.path)
    for g, r in zip(gp, o.path):
        assert g["kind"] == r["kind"]
        assert g["beta"] == pytest.approx(r["beta"], rel=1e-7, abs=1e-7)
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-7, atol=1e-8)
    assert h.state()["evals"][:2] == list(o.evals)


def test_flow_cell_is_not_batched():
    obs = wl.obs_grid(7)
    h = native.Handle([16], K, obs, np.zeros(49), 0.045, corr_len=LC, precision=native.SMC_MIXED, cov="matern",
                      bc="flow_cell")
    with pytest.raises(native.SmcError):
        native.Batch([h])
