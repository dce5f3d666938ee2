"""One small launch of the likelihood kernel, for profiler captures (ncu) of a single kernel.

python -m paper_1709_09763_gb300.profile_case [--inv-h 64] [--J 304] [--launches 2] [--precision mixed]
                                             [--block 0] [--workload mls2mc_mixed_h8_64]
                                             [--train-steps 0 --batch 8192]
Uses a workload's KL settings (terms, covariance), source, boundary conditions, observation grid
and data with seeded particles (default: the MLS^2MC workload); --block forces the threads per
particle (0: the library default; -512 at 1/h = 64: the compact form; -1024 at 1/h = 128: the
two-CTA form). --train-steps S instead runs S surrogate Adam steps (after three untimed ones) on
minibatches of --batch pairs drawn from 40,000 seeded pairs, with the workload's K and
observation count, and prints the wall time per step.
"""
import argparse
import json
import os

import numpy as np

from . import build, native
from . import workloads as wl


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--inv-h", type=int, default=64)
    ap.add_argument("--J", type=int, default=304)
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--workload", default="mls2mc_mixed_h8_64", choices=sorted(wl.WORKLOADS))
    ap.add_argument("--train-steps", type=int, default=0)
    ap.add_argument("--batch", type=int, default=8192)
    a = ap.parse_args()
    import torch
    build.build()
    w = wl.WORKLOADS[a.workload]
    if a.train_steps > 0:
        train_case(w, a)
        return
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "tests", "golden", f"data_{w.name}.json")) as f:
        d = json.load(f)
    prec = native.SMC_MIXED if a.precision == "mixed" else native.SMC_FP64
    h = native.Handle([a.inv_h], w.K, wl.obs_grid(w.obs_per_side), d["y"], d["sigma"], corr_len=w.corr_len,
                      precision=prec, cov=w.cov, source=w.source, bc=w.bc)
    if a.block:
        h.set_block_size(0, a.block)
    th = torch.from_numpy(wl.particles(a.J, w.K, 5)).cuda()
    G = torch.empty((a.J, w.n_obs), dtype=torch.float64, device="cuda")
    Phi = torch.empty(a.J, dtype=torch.float64, device="cuda")
    it = torch.empty(a.J, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(a.launches):
        h.eval_likelihood_device(0, a.J, th.data_ptr(), G.data_ptr(), Phi.data_ptr(), it.data_ptr(), s)
    torch.cuda.synchronize()
    its = it.cpu().numpy()
    assert (its > 0).all(), "non-converged solve"
    print(json.dumps({"workload": w.name, "inv_h": a.inv_h, "J": a.J, "block": a.block,
                      "mean_iters": float(np.mean(its))}))


def train_case(w, a):
    """Surrogate training steps of one level's network on seeded random pairs."""
    import time
    import torch
    obs = wl.obs_grid(w.obs_per_side)
    n_obs = obs.shape[0]
    h = native.Handle([a.inv_h], w.K, obs, np.zeros(n_obs), 1.0, corr_len=w.corr_len, J=a.batch,
                      precision=native.SMC_MIXED, surrogate=1)
    rng = np.random.default_rng(0)
    h.surrogate_add_pairs(0, rng.standard_normal((40000, w.K)), 1e-3 * rng.standard_normal((40000, n_obs)))
    h.surrogate_train(0, 3, a.batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = h.surrogate_train(0, a.train_steps, a.batch)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({"workload": w.name, "K": w.K, "n_obs": n_obs, "batch": a.batch, "steps": a.train_steps,
                      "ms_per_step": 1e3 * dt / a.train_steps, "loss": loss}))


if __name__ == "__main__":
    main()
