"""Write the synthetic data vectors y (one JSON file per workload) using only the oracle.

Sec. 5: the true parameter is drawn from the (discretised) prior and the data are
its forward response plus Gaussian noise. Here theta_true and the noise draw come
from the seeded generators of the workloads module; the forward response is the
oracle's FP64 P1 solution on the data mesh (finer than every sampler level), and
sigma is the workload's absolute noise level (Examples 5.1, 5.2) or noise_frac
times the largest nodal value of that solution.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np                                     # noqa: E402

from oracle import fem, kl, matern                     # noqa: E402
from paper_1709_09763_gb300 import workloads as wl     # noqa: E402


def make(w):
    N = w.inv_h_data
    th = wl.theta_true(w)
    if w.cov == "matern":
        u = matern.field(N, th, w.corr_len, w.variance, w.K)
    else:
        u = th @ kl.kl_table(N, w.corr_len, w.variance, w.K)
    f = fem.nine_sources if w.source == "nine" else None
    if w.bc == "flow_cell":
        p = fem.solve_flow_cell(N, np.exp(u))
    else:
        p = fem.solve(N, np.exp(u), f)
    obs = wl.obs_grid(w.obs_per_side)
    G = fem.observation_operator(N, obs) @ p
    sigma = w.sigma_abs if w.sigma_abs > 0 else w.noise_frac * np.abs(p).max()
    y = G + sigma * wl.noise(w)
    return dict(workload=w.name, inv_h_data=N, theta_true=th.tolist(), sigma=float(sigma),
                y=y.tolist(), G_data=G.tolist())


if __name__ == "__main__":
    names = sys.argv[1:] or list(wl.WORKLOADS)
    for name in names:
        d = make(wl.WORKLOADS[name])
        with open(os.path.join(HERE, f"data_{name}.json"), "w") as f:
            json.dump(d, f, indent=1)
        print(name, "sigma", d["sigma"])
