"""The paper's Example 5.1/5.2 workload on the GPU path against the FP64 oracle: Matern KL table,
the nine-source load vector inside the solve (every solve form: shared memory, compact, device
memory at 1/128), and the random-walk sampler's update path and particles on the FP64 path."""
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
W = wl.WORKLOADS["example_5_1"]
# compiled threads-per-particle variants (negative: compact forms; -1024 at 1/128: the two-CTA form)
SIZES = {native.SMC_MIXED: {8: [64, 32], 16: [128, 64], 32: [256, 512, -256], 64: [512, 1024, -512], 128: [1024, -1024]},
         native.SMC_FP64: {8: [64], 16: [128, 256], 32: [256, 512]}}


def _data(name):
    with open(os.path.join(GOLD, f"data_{name}.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _handle(levels, prec, **kw):
    d = _data(W.name)
    return native.Handle(levels, W.K, wl.obs_grid(W.obs_per_side), d["y"], d["sigma"], corr_len=W.corr_len,
                         precision=prec, cov="matern", source="nine", **kw), d


def _rel(a, b):
    return np.max(np.abs(a - b), axis=-1) / np.max(np.abs(b), axis=-1)


def test_matern_kl_table_matches_oracle():
    h, _ = _handle(list(W.inv_h), native.SMC_MIXED)
    for l, N in enumerate(W.inv_h):
        psi, lam = h.kl_table(l, N)
        assert np.allclose(lam, omat.eigenvalues(W.corr_len, 1.0, W.K), rtol=1e-11)
        assert np.abs(psi - omat.kl_table(N, W.corr_len, 1.0, W.K)).max() < 1e-12


@pytest.mark.parametrize("prec", [native.SMC_MIXED, native.SMC_FP64])
def test_example_5_1_likelihood_parity(prec):
    """G with the Matern field and the nine sources: 1e-6 (mixed) / 1e-10 (FP64) of the oracle at
    every level of the hierarchy (FP64 up to 1/32), every compiled block size of the mixed path."""
    levels = list(W.inv_h) if prec == native.SMC_MIXED else [8, 16, 32]
    tol = 1e-6 if prec == native.SMC_MIXED else 1e-10
    h, d = _handle(levels, prec)
    obs = wl.obs_grid(W.obs_per_side)
    theta = wl.particles(5, W.K, 515)
    for l, N in enumerate(levels):
        lv = ofwd.Level(N, W.corr_len, 1.0, W.K, obs, f=ofem.nine_sources, cov="matern")
        Gr = lv.G_batch(theta)
        for T in SIZES[prec][N]:
            h.set_block_size(l, T)
            G, Phi = h.eval_likelihood(l, theta)
            assert _rel(G, Gr).max() < tol, (N, T)
        h.set_block_size(l, 0)
        G, Phi = h.eval_likelihood(l, theta)
        Phir = potential(Gr, np.array(d["y"]), d["sigma"])
        assert np.allclose(Phi, Phir, rtol=50 * tol)


def test_example_5_1_compact_forms_bit_identical():
    """The compact solve forms read the load vector like the shared-memory forms: same bits."""
    h, _ = _handle([32, 64], native.SMC_MIXED)
    theta = wl.particles(700, W.K, 516)
    for l, T in ((0, 256), (1, 512)):
        out = []
        for B in (T, -T):
            h.set_block_size(l, B)
            out.append(h.eval_likelihood(l, theta)[1])
        assert np.array_equal(out[0], out[1])
        h.set_block_size(l, 0)


def test_example_5_1_rwm_sampler_matches_oracle_path():
    """FP64 path, levels 1/8 and 1/16, Matern field, nine sources, one random-walk step per update
    (covariance 2.38^2 / K): the same update path, evaluation counts and particles as the oracle."""
    K, J = W.K, 400
    obs = wl.obs_grid(W.obs_per_side)
    d = _data(W.name)
    y, sigma = np.array(d["y"]), d["sigma"]
    lv = [ofwd.Level(N, W.corr_len, 1.0, K, obs, f=ofem.nine_sources, cov="matern") for N in (8, 16)]
    kw = dict(J_tilde=50, n_mcmc=1, s_pcn=2.38 / math.sqrt(K), seed=43)
    h = native.Handle([8, 16], K, obs, y, sigma, corr_len=W.corr_len, J=J, precision=native.SMC_FP64, rtol=1e-13,
                      cov="matern", source="nine", proposal="rwm", **kw)
    h.run()
    ev = lambda l, th: potential(lv[l].G_batch(th), y, sigma)
    o = smc.Sampler(ev, 2, K, J, proposal="rwm", **kw).run()
    gp = h.path()
    assert len(gp) == len(o.path)
    for g, r in zip(gp, o.path):
        assert g["kind"] == r["kind"]
        assert g["beta"] == pytest.approx(r["beta"], rel=1e-7, abs=1e-7)
        assert g["accept_rate"] == pytest.approx(r["accept"], abs=1e-12)
    th, _ = h.particles()
    assert np.allclose(th, o.theta, rtol=1e-7, atol=1e-8)
    assert h.state()["evals"][:2] == list(o.evals)
    assert 0.05 < np.mean([g["accept_rate"] for g in gp]) < 0.9



def test_mls2mc_and_single_level_smc_agree_on_example_5_1():
    """Both samplers target the posterior of the finest level: MLS^2MC on 1/8, 1/16, 1/32 and
    single-level SMC on 1/32 (Example 5.1 data, random-walk kernel) agree in every posterior mean
    within 4 standard errors of the difference, estimated from 10 seeded runs of each."""
    d = _data(W.name)
    obs = wl.obs_grid(W.obs_per_side)
    J, R = 2500, 10
    res = {}
    for name, levels in (("mls2mc", [8, 16, 32]), ("smc", [32])):
        means = []
        for r in range(R):
            h = native.Handle(levels, W.K, obs, d["y"], d["sigma"], corr_len=W.corr_len, J=J, n_mcmc=5,
                              s_pcn=2.38 / math.sqrt(W.K), precision=native.SMC_MIXED, seed=1000 + 7 * r,
                              cov="matern", source="nine", proposal="rwm")
            h.run()
            st = h.state()
            assert st["beta"] == 1.0 and st["level"] == len(levels) - 1
            means.append(h.posterior_moments()[0])
            h.close()
        res[name] = np.array(means)
    a, b = res["mls2mc"], res["smc"]
    se = np.sqrt(a.var(0, ddof=1) / R + b.var(0, ddof=1) / R)
    assert np.all(np.abs(a.mean(0) - b.mean(0)) < 4 * se + 1e-3), (a.mean(0), b.mean(0), se)
