"""Posterior moments of the GPU sampler against brute-force quadrature (K = 2 FEM problem).

tests/golden/quad_k2_h16.json holds the exact posterior mean and variance of the discretised
problem on 1/h = 16 (oracle FEM, trapezoid grid, grid error ~1e-11). R seeded replicates of the
mixed-precision MLS^2MC sampler (levels 1/8, 1/16), plain and with the surrogate screen forced on
every level, with pCN and with the covariance-shaped random walk (step 2.38 / sqrt(2)), must give replicate-averaged posterior means and variances within 3 Monte Carlo
standard errors of it (the standard error estimated from the replicate spread). With R = 32 the
deviation over its estimated standard error follows Student's t with 31 degrees of freedom: a
correct sampler exceeds 3 in one of the four comparisons of a run with probability 2.1 %."""
import json
import os

import numpy as np
import pytest

from paper_1709_09763_gb300 import native

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "quad_k2_h16.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


@pytest.mark.parametrize("surrogate,proposal,step", [(0, "pcn", 0.3), (2, "pcn", 0.3), (0, "rwm_cov", 1.68),
                                                     (2, "rwm_cov", 1.68)])
def test_sampler_matches_quadrature_within_3_se(surrogate, proposal, step):
    q = json.load(open(GOLD))
    R = 32
    means, vars_ = [], []
    for r in range(R):
        h = native.Handle([8, 16], 2, np.array(q["obs"]), q["y"], q["sigma"], corr_len=q["corr_len"], J=2000,
                          J_tilde=100, n_mcmc=5, s_pcn=step, precision=native.SMC_MIXED, seed=1000 + r,
                          surrogate=surrogate, proposal=proposal)
        h.run()
        m, v, _ = h.posterior_moments()
        means.append(m)
        vars_.append(v)
        h.close()
    means, vars_ = np.array(means), np.array(vars_)
    for est, ref, err in ((means, q["mean"], q["quad_err_mean"]), (vars_, q["var"], q["quad_err_var"])):
        se = est.std(axis=0, ddof=1) / np.sqrt(R)
        dev = np.abs(est.mean(axis=0) - np.array(ref))
        assert np.all(dev <= 3.0 * se + np.array(err)), (est.mean(axis=0), ref, se)
