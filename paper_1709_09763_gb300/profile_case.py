"""One small launch of the likelihood kernel, for profiler captures (ncu) of a single kernel.

python -m paper_1709_09763_gb300.profile_case [--inv-h 64] [--J 304] [--launches 2] [--precision mixed]
                                             [--block 0] [--workload mls2mc_mixed_h8_64]
Uses a workload's KL settings (terms, covariance), source, boundary conditions, observation grid
and data with seeded particles (default: the MLS^2MC workload); --block forces the threads per
particle (0: the library default; -512 at 1/h = 64: the compact form).
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
    a = ap.parse_args()
    import torch
    build.build()
    w = wl.WORKLOADS[a.workload]
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


if __name__ == "__main__":
    main()
