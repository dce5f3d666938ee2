"""Synthetic workloads: sizes, seeds and seeded input draws (no arithmetic of the method).

The paper's experiments (Sec. 5) use synthetic data: a true parameter drawn from
the prior and observations of its forward response plus Gaussian noise. The
workloads below fix the shapes of those experiments for this library: level
hierarchy, KL truncation, observation grid, particle count and Markov steps.
This module only draws seeded standard-normal inputs and lists coordinates; the
data vector y itself is produced by solving the forward problem, which is not
done here.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    inv_h: tuple            # level hierarchy, 1/h per level, coarse to fine
    inv_h_data: int         # mesh used to synthesise y (finer than every level)
    K: int                  # KL terms (N_sto)
    corr_len: float         # correlation length of the exponential covariance
    obs_per_side: int       # observation grid: points (i/(n+1), j/(n+1)), i, j = 1..n
    J: int                  # particles
    n_mcmc: int             # pCN steps per update
    s_pcn: float = 0.2
    tau_star: float = 1.0
    J_tilde: int = 100
    variance: float = 1.0
    seed_true: int = 1
    seed_noise: int = 2
    seed_sampler: int = 3
    precision: str = "fp64"   # "fp64" or "mixed"
    noise_frac: float = 0.01  # sigma = noise_frac * max |p_data| (unless sigma_abs is set)
    sigma_abs: float = 0.0    # > 0: the noise standard deviation itself
    cov: str = "sep_exp"      # prior covariance: "sep_exp" (separable exponential) or "matern" (nu = 3/2)
    source: str = "one"       # source term: "one" (f = 1) or "nine" (the nine sources of Example 5.1)
    proposal: str = "pcn"     # Markov kernel: "pcn" or "rwm" (random walk, step s_pcn)
    bc: str = "dirichlet"     # boundary conditions: "dirichlet" or "flow_cell" (Example 5.3)
    tau_min: float = 0.0      # > 0: the update scheme u' (adaptive maximum level)

    @property
    def n_obs(self):
        return self.obs_per_side ** 2


WORKLOADS = {
    # single-level SMC, plain FP64, h = 1/16
    "smc_fp64_h16": Workload("smc_fp64_h16", (16,), 64, 16, 0.3, 7, 1000, 5,
                             seed_true=1, seed_noise=2, seed_sampler=3, precision="fp64"),
    # MLS^2MC, 4 levels h = 1/8 .. 1/64, K = 32, J = 4000, mixed precision
    "mls2mc_mixed_h8_64": Workload("mls2mc_mixed_h8_64", (8, 16, 32, 64), 256, 32, 0.1, 7,
                                   4000, 5, seed_true=11, seed_noise=12, seed_sampler=13,
                                   precision="mixed"),
    # surrogate-screened MLS^2MC, 5 levels h = 1/8 .. 1/128, K = 64, J = 8000, 10 pCN steps
    "da_mixed_h8_128": Workload("da_mixed_h8_128", (8, 16, 32, 64, 128), 512, 64, 0.1, 7,
                                8000, 10, seed_true=21, seed_noise=22, seed_sampler=23,
                                precision="mixed"),
    # large: 5 levels h = 1/16 .. 1/256, K = 128, correlation length 0.05, 12 x 12 observations,
    # J = 16384, 10 pCN steps
    "large_mixed_h16_256": Workload("large_mixed_h16_256", (16, 32, 64, 128, 256), 1024, 128, 0.05,
                                    12, 16384, 10, seed_true=31, seed_noise=32, seed_sampler=33,
                                    precision="mixed"),
    # the paper's Example 5.1 (Sec. 5): 5 levels h = 1/8 .. 1/128, Matern prior (lc = 0.65, nu = 3/2)
    # with N_sto = 10, nine smoothed point sources, 25 observations, Gamma = 0.07^2 I, one
    # random-walk step (proposal covariance 2.38^2 / N_sto I) per update, J = 2500, tau* = 1
    "example_5_1": Workload("example_5_1", (8, 16, 32, 64, 128), 256, 10, 0.65, 5, 2500, 1,
                            s_pcn=2.38 / 10 ** 0.5, seed_true=41, seed_noise=42, seed_sampler=43,
                            precision="mixed", sigma_abs=0.07, cov="matern", source="nine", proposal="rwm"),
    # Example 5.2: the same problem and data draw with Gamma = 0.035^2 I
    "example_5_2": Workload("example_5_2", (8, 16, 32, 64, 128), 256, 10, 0.65, 5, 2500, 1,
                            s_pcn=2.38 / 10 ** 0.5, seed_true=41, seed_noise=42, seed_sampler=53,
                            precision="mixed", sigma_abs=0.035, cov="matern", source="nine", proposal="rwm"),
    # the paper's Example 5.3 (flow cell) at reduced size: levels 1/16 .. 1/64 (the paper: to 1/256),
    # Matern prior lc = 0.1 with 64 terms (the paper: 320, see example_5_3_full; its m0 = 2 is
    # irrelevant since f = 0),
    # 49 observations, Gamma = 0.045^2 I, one random-walk step per update, scheme u' with
    # tau_min = 0.001, J = 1000
    "example_5_3": Workload("example_5_3", (16, 32, 64), 128, 64, 0.1, 7, 1000, 1,
                            s_pcn=2.38 / 64 ** 0.5, seed_true=71, seed_noise=72, seed_sampler=73,
                            precision="mixed", sigma_abs=0.045, cov="matern", proposal="rwm",
                            bc="flow_cell", tau_min=0.001),
    # Example 5.3 at the paper's size: levels 1/16 .. 1/256, Matern prior lc = 0.1 with
    # N_sto = 320 terms, 49 observations, Gamma = 0.045^2 I, one random-walk step (covariance
    # 2.38^2 / 320 I) per update, scheme u' with tau_min = 0.001, J = 1000
    "example_5_3_full": Workload("example_5_3_full", (16, 32, 64, 128, 256), 512, 320, 0.1, 7, 1000, 1,
                                 s_pcn=2.38 / 320 ** 0.5, seed_true=81, seed_noise=82, seed_sampler=83,
                                 precision="mixed", sigma_abs=0.045, cov="matern", proposal="rwm",
                                 bc="flow_cell", tau_min=0.001),
}


def obs_grid(n):
    """Points (i/(n+1), j/(n+1)) for i, j = 1..n, row-major in j. n = 7 gives (i/8, j/8)."""
    pts = [((i + 1) / (n + 1), (j + 1) / (n + 1)) for j in range(n) for i in range(n)]
    return np.array(pts, dtype=np.float64)


def standard_normals(shape, seed):
    """Seeded N(0, 1) draws (numpy PCG64); used for theta_true, noise and test particles."""
    return np.random.default_rng(seed).standard_normal(shape)


def theta_true(w: Workload):
    return standard_normals((w.K,), w.seed_true)


def noise(w: Workload):
    return standard_normals((w.n_obs,), w.seed_noise)


def particles(J, K, seed):
    """Test/bench particle batch theta ~ N(0, I_K), shape (J, K)."""
    return standard_normals((J, K), seed)


def batched_uneven(n_problems=64, seed=7, max_inv_h=64, j_range=(500, 8000)):
    """Independent problems of uneven size: finest mesh 1/h drawn from {16, 32, 64} (and 128 when
    max_inv_h allows), hierarchy from 1/8 up to it, K from {16, 32, 64} (correlation length 0.3,
    0.1, 0.1), J log-uniform in j_range (default [500, 8000]); problem p uses theta_true seed
    100 + p and noise seed 200 + p. Returns a list of dicts (levels, K, corr_len, J, seed_true,
    seed_noise)."""
    rng = np.random.default_rng(seed)
    finest = [h for h in (16, 32, 64, 128) if h <= max_inv_h]
    out = []
    for p in range(n_problems):
        f = int(rng.choice(finest))
        K = int(rng.choice([16, 32, 64]))
        lc = 0.3 if K == 16 else 0.1
        J = int(round(np.exp(rng.uniform(np.log(j_range[0]), np.log(j_range[1])))))
        levels = tuple(h for h in (8, 16, 32, 64, 128) if h <= f)
        out.append(dict(levels=levels, K=K, corr_len=lc, J=J, seed_true=100 + p, seed_noise=200 + p))
    return out
