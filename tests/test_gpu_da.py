"""Delayed-acceptance pCN with the trained surrogate leaves the posterior unchanged and saves exact
solves (screen forced on every level: surrogate = 2). R = 16 seeded replicates of the plain and the
surrogate-screened MLS^2MC sampler on the same FEM problem: for every posterior mean and variance the
Welch t statistic of the two arms' replicate means stays below the two-sided critical value of a
family-wise false-alarm rate of 1e-3 (Bonferroni over the 2K moments; about 4.9 standard errors at
these degrees of freedom), and the screened sampler solves fewer exact forward problems per pCN
proposal."""
import numpy as np
import pytest

from oracle import forward as ofwd
from paper_1709_09763_gb300 import native
from paper_1709_09763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _problem():
    K = 8
    obs = wl.obs_grid(7)
    lv = ofwd.Level(32, 0.3, 1.0, K, obs)
    th_true = np.random.default_rng(11).standard_normal(K)
    G = lv.G(th_true)
    sigma = 0.02 * np.abs(G).max()
    y = G + sigma * np.random.default_rng(12).standard_normal(obs.shape[0])
    return K, obs, y, sigma


def _run(surrogate, seed, K, obs, y, sigma, proposal="pcn"):
    h = native.Handle([8, 16, 32], K, obs, y, sigma, corr_len=0.3, J=1500, J_tilde=100, n_mcmc=5,
                      s_pcn=0.3 if proposal == "pcn" else 2.38 / np.sqrt(K), precision=native.SMC_MIXED, seed=seed,
                      surrogate=surrogate, surrogate_train_steps=150, proposal=proposal)
    h.run()
    m, v, lz = h.posterior_moments()
    path = h.path()
    st = h.state()
    h.close()
    return m, v, lz, path, st


@pytest.mark.parametrize("proposal", ["pcn", "rwm"])
def test_delayed_acceptance_same_posterior_fewer_solves(proposal):
    """With the pCN kernel, and with the random walk (whose prior ratio enters stage 1)."""
    stats = pytest.importorskip("scipy.stats")
    K, obs, y, sigma = _problem()
    R = 16
    plain = [_run(0, 100 + r, K, obs, y, sigma, proposal) for r in range(R)]
    da = [_run(2, 100 + r, K, obs, y, sigma, proposal) for r in range(R)]
    for idx in (0, 1):   # means, variances
        a = np.array([p[idx] for p in plain])
        b = np.array([d[idx] for d in da])
        va, vb = a.var(axis=0, ddof=1) / R, b.var(axis=0, ddof=1) / R
        se = np.sqrt(va + vb)
        dof = (va + vb) ** 2 / (va ** 2 / (R - 1) + vb ** 2 / (R - 1))          # Welch-Satterthwaite
        crit = stats.t.ppf(1.0 - 1e-3 / (2 * 2 * K), dof)
        z = np.abs(a.mean(axis=0) - b.mean(axis=0)) / se
        print(f"{proposal} moment {idx}: max |t| {z.max():.2f}, critical {crit.min():.2f}")
        assert np.all(z <= crit), (idx, a.mean(0), b.mean(0), se, crit)
    # the screen is active: some updates ran stage 1, and it rejected part of the proposals
    rates = [p["da_stage1_rate"] for d in da for p in d[3] if p["da_stage1_rate"] >= 0]
    assert len(rates) > 0 and np.mean(rates) < 0.9
    # exact solves per pCN proposal: 1 per level for the plain sampler, fewer with the screen
    def solves_per_update(run):
        total = sum(run[4]["evals"][:3])
        props = sum(1 for _ in run[3])
        return total / props
    assert np.mean([solves_per_update(d) for d in da]) < np.mean([solves_per_update(p) for p in plain])


def test_cost_gate_follows_measured_costs():
    """surrogate = 1 never screens a level whose measured exact solve of J particles costs at most 8
    surrogate passes; above that it screens from the first update whose own 5 sweeps of exact solves,
    with those already run on the level, cost twice the first training round (50 Adam steps, each
    estimated as 4 forward passes of its minibatch). Single-level SMC on 1/h = 64 with J = 1500 and
    minibatches of 1500 (every update an ITU on that level): the gate's decision and the first
    screened update follow the measured times, and the sampler reaches beta = 1."""
    K, obs, y, sigma = _problem()
    J = 1500
    h = native.Handle([64], K, obs, y, sigma, corr_len=0.3, J=J, n_mcmc=5, s_pcn=0.3,
                      precision=native.SMC_MIXED, seed=7, surrogate=1, surrogate_batch=J)
    h.run()
    path = h.path()
    assert all(p["kind"] == "ITU" for p in path)
    dec, t_solve, t_pred = h.surrogate_gate(0)
    assert t_solve > 0 and t_pred > 0
    assert (dec < 0) == (t_solve <= 8 * t_pred)
    screened = [p["da_stage1_rate"] >= 0 for p in path]
    assert any(screened) == (dec > 0)
    # exact-solve ms after each update, and with the next update's 5 sweeps
    spent = [p["evals_per_level"][0] * t_solve / J for p in path]
    threshold = 2 * 50 * 4 * t_pred
    if dec > 0:
        u = screened.index(True)
        if u >= 1:   # at the start of update u the level had spent spent[u - 1] (its updates add solves only in moves)
            assert spent[u - 1] + 5 * t_solve >= threshold
        if u >= 2:   # and at the start of update u - 1, spent[u - 2]
            assert spent[u - 2] + 5 * t_solve < threshold
    elif dec == 0:
        assert len(path) < 2 or spent[-2] + 5 * t_solve < threshold
    assert h.state()["beta"] == 1.0


def test_gate_forced_and_unmeasured():
    """surrogate = 2 screens without a measurement (zero times); a plain sampler never measures."""
    K, obs, y, sigma = _problem()
    h = native.Handle([8, 16], K, obs, y, sigma, corr_len=0.3, J=300, n_mcmc=2, s_pcn=0.3,
                      precision=native.SMC_MIXED, seed=3, surrogate=0)
    h.run()
    assert h.surrogate_gate(0) == (0, 0.0, 0.0) and h.surrogate_gate(1) == (0, 0.0, 0.0)
    with pytest.raises(native.SmcError):
        h.surrogate_gate(2)


def test_screened_sampler_is_reproducible():
    """The screened sampler is deterministic for a given seed: stage-1 survivors are compacted in
    particle order, so the exact solves and the training pairs they add to the surrogate's set come
    in the same order on every run (bit-identical posterior moments and evidence)."""
    K, obs, y, sigma = _problem()
    a = _run(2, 77, K, obs, y, sigma)
    b = _run(2, 77, K, obs, y, sigma)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    assert a[4]["evals"] == b[4]["evals"]
