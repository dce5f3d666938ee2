"""Benchmark of the MLS^2MC likelihood hot path on GB300.

Workload: the MLS^2MC configuration of 4 levels h = 1/8, 1/16, 1/32, 1/64, K = 32 KL
terms (correlation length 0.1), 49 observations on the 7 x 7 grid, J = 4000 particles,
mixed precision (FP32 multigrid-PCG with extended-precision refinement). One step is
one pass of the hot path over the particle batch: on every level a tempering update and,
below the finest level, a bridging step to the next level, each with 5 pCN sweeps -- the
likelihood G_l(theta), Phi_l(theta) (KL field, P1 solve, observation gather, Gaussian
misfit) of every particle and proposal, the adaptive increments, resampling and moves.

value: likelihood evaluations per second over the whole job (all levels, all ranks),
inputs resident in device memory, L2 flushed between steps. e2e: the same step through
the host-pointer C-ABI call (theta copied in from pinned host memory, G and Phi copied
out every step). Multi-GPU: independent replicas per rank (no data-path collective).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "mls2mc_mixed_h8_64"


# DRAM bytes per particle of the 1/64 solve kernels by threads per particle (kappa in, G and Phi
# out), measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum) on one launch of the same
# kernel and scaled by the particle count (the traffic is per particle: nothing is shared between
# blocks); None where no capture of the current build exists
FEM64_DRAM_BYTES_PER_PARTICLE = {512: None, 1024: None, -512: (20.061184e6 + 4.715776e6) / 608}


def solve_kernel_name(N, T):
    """Name of the solve kernel that runs level 1/h = N with T threads per particle."""
    return f"fem_eval_compact<{N},{-T}>" if T < 0 else f"fem_eval_kernel<float,{N},{T}>"


def algorithmic_flops_per_eval(N, K, iters, passes, synthesis=False):
    """FP32 operations of one likelihood evaluation on level 1/h = N, counted from the algorithm.

    Per fine interior node and CG iteration: V(1,1) fine-level work (red/black smoothing
    before and after: 2 x (0.5 x 1 + 0.5 x 10), residual 11, restriction 2, prolongation
    1.5) = 24.5, coarse levels 1/3 of that, CG vector work 22 -> 54.7. Per refinement pass:
    the residual update in double-float arithmetic, ~100 FP32 operations per node. Set-up:
    coefficients ~10 per node, and with synthesis=True the KL synthesis 2*K*E and exp E (on the
    mixed path the synthesis runs in the tensor-core GEMM, not in the solve kernel).
    """
    n = (N - 1) ** 2
    E = 2 * N * N
    per_iter = (24.5 * 4.0 / 3.0 + 22.0) * n
    synth = 2.0 * K * E + E if synthesis else 0.0
    return iters * per_iter + passes * 100.0 * n + synth + 10.0 * (N + 1) ** 2


def algorithmic_smem_bytes_per_eval(N, iters, passes):
    """Shared-memory bytes one evaluation on level 1/h = N moves, counted from the solve's algorithm
    (4-byte words; the block reductions' broadcast reads are not counted).

    Per fine node and CG iteration: a black node loads 9 words (4 weights, 4 neighbours, its inverse
    diagonal) and stores 1 in the black pre-sweep, loads 13 (the same plus 4 coarse values) and
    stores 1 in the post-sweep with the prolongation, stores p once and loads 8 in A p; a red node
    loads 8 and stores 1 for its residual, loads 9 in the red post-sweep, stores p, loads 8 in A p,
    loads 1 and stores 1 for the next red pre-sweep: 31 words on average. The coarse levels add
    about 26 words per coarse node (a quarter of the fine nodes per level): 8.7 more per fine node.
    Per refinement pass: 18 words per node (d published, A d in edge form, x and r pairs). Set-up:
    16 words per node (kappa staging, coefficients, coarsening)."""
    n = (N - 1) ** 2
    return 4.0 * n * (iters * (31.0 + 8.7) + passes * 18.0 + 16.0)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max_over_ranks(values, dist=None, device="cpu"):
    """Every rank gets the element-wise max of `values` over all ranks (identity on one rank)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job units per second: all ranks' units over the slowest rank's time (weak scaling)."""
    return units_per_rank * world / (ms_max * 1e-3)


def load_data(name=WORKLOAD):
    with open(os.path.join(ROOT, "tests", "golden", f"data_{name}.json")) as f:
        return json.load(f)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(job):
    """One host process of the oracle timing: FP64 evaluations of the workload's particles, round
    robin over its levels, for `seconds` (or `count` particles per level). Runs in a spawned process
    with one BLAS thread."""
    name, seconds, count, offset = job
    from oracle import forward as ofwd
    from paper_1709_09763_gb300 import workloads as wl
    w = wl.WORKLOADS[name]
    d = load_data(name)
    obs = wl.obs_grid(w.obs_per_side)
    levels = [ofwd.Level(N, w.corr_len, w.variance, w.K, obs) for N in w.inv_h]
    theta = wl.particles(64, w.K, 777 + offset)
    t0 = time.perf_counter()
    n = 0
    while True:
        for lv in levels:
            ofwd.potential(lv.G(theta[n % 64]), d["y"], d["sigma"])
            n += 1
        if (count is not None and n >= count * len(levels)) or (count is None and time.perf_counter() - t0 > seconds):
            break
    return n, time.perf_counter() - t0


class OraclePool:
    """Spawned host processes (one BLAS thread each) that run the FP64 oracle; spawn, not fork,
    because the parent has a CUDA context."""

    def __init__(self, procs):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs)
        # warm the workers (imports, KL tables) outside any timing
        self.pool.map(_oracle_worker, [(WORKLOAD, 0.0, 1, i) for i in range(procs)])

    def run(self, seconds=None, count=None):
        res = self.pool.map(_oracle_worker, [(WORKLOAD, seconds, count, i) for i in range(self.procs)])
        return sum(r[0] for r in res), max(r[1] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(seconds=6.0):
    """The FP64 oracle timed on the host: on one core, and on every host core (one process per
    core, each evaluating its own particles round robin over the 4 levels)."""
    cores = host_cores()
    out = {"unit": "evals/s", "kind": "oracle"}
    for label, procs in (("single_core", 1), ("all_cores", cores)):
        pool = OraclePool(procs)
        n, dt = pool.run(seconds=seconds)
        pool.close()
        out[label] = {"value": n / dt, "cores": procs,
                      "sample": f"{n} FP64 oracle evaluations (levels 1/8..1/64 round robin, sparse direct "
                                f"solve) in {dt:.1f} s on {procs} host core(s)"}
    out["value"] = out["all_cores"]["value"]
    out["cores"] = cores
    out["sample"] = out["all_cores"]["sample"]
    return out


def run_reference(args, rank):
    """The oracle as the reference arm: each step a bounded sample of the workload on every host
    core (one spawned process per core, one particle per level each)."""
    if rank != 0:
        return
    from paper_1709_09763_gb300 import workloads as wl
    w = wl.WORKLOADS[WORKLOAD]
    cores = host_cores()
    pool = OraclePool(cores)
    for _ in range(args.warmup):
        pool.run(count=1)
    t0 = time.perf_counter()
    evals = 0
    for _ in range(args.steps):
        evals += pool.run(count=1)[0]
    dt = (time.perf_counter() - t0) / args.steps
    pool.close()
    per_step = evals / args.steps
    value = per_step / dt
    sample = f"{cores} particles x {len(w.inv_h)} levels per step, one host process per core"
    line = {"impl": "reference", "metric": "likelihood evals/s per mesh level", "value": value,
            "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels_inv_h": list(w.inv_h), "K": w.K, "n_obs": w.n_obs,
                       "J": w.J, "precision": "fp64 oracle", "sample": sample},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_measurement(native, wl, torch, dev, reps=5, n_problems=64, max_inv_h=128, j_range=(500, 8000)):
    """n_problems independent problems of uneven size (finest 1/h in {16, 32, 64, 128} up to
    max_inv_h, J log-uniform in j_range), each evaluating its J particles on its finest level:
    sequential per-problem launches against one batch (persistent launch per level size) replayed
    as a CUDA graph. Data: y = G(theta_true) on the finest level + 1 % noise, from the library."""
    specs = wl.batched_uneven(n_problems=n_problems, max_inv_h=max_inv_h, j_range=j_range)
    stream = torch.cuda.Stream(dev)
    obs = wl.obs_grid(7)
    hs, th, ph, it = [], [], [], []
    with torch.cuda.stream(stream):
        for sp in specs:
            h0 = native.Handle(sp["levels"], sp["K"], obs, np.zeros(49), 1.0, corr_len=sp["corr_len"],
                               precision=native.SMC_MIXED, stream=stream.cuda_stream)
            tt = wl.standard_normals((1, sp["K"]), sp["seed_true"])
            G, _ = h0.eval_likelihood(len(sp["levels"]) - 1, tt)
            h0.close()
            sigma = 0.01 * float(np.abs(G).max())
            y = G[0] + sigma * wl.standard_normals((49,), sp["seed_noise"])
            h = native.Handle(sp["levels"], sp["K"], obs, y, sigma, corr_len=sp["corr_len"],
                              precision=native.SMC_MIXED, stream=stream.cuda_stream)
            hs.append(h)
            th.append(torch.from_numpy(wl.particles(sp["J"], sp["K"], 5000 + len(hs))).to(dev))
            ph.append(torch.empty(sp["J"], dtype=torch.float64, device=dev))
            it.append(torch.empty(sp["J"], dtype=torch.int32, device=dev))
    levels = [len(sp["levels"]) - 1 for sp in specs]
    counts = [sp["J"] for sp in specs]
    total = sum(counts)
    s = stream.cuda_stream

    def sequential():
        for h, l, n, t, p, i in zip(hs, levels, counts, th, ph, it):
            h.eval_likelihood_device(l, n, t.data_ptr(), 0, p.data_ptr(), i.data_ptr(), s)
    b = native.Batch(hs)

    def batched():
        b.eval(levels, counts, [t.data_ptr() for t in th], [p.data_ptr() for p in ph], [i.data_ptr() for i in it],
               s, True)

    def timed(fn):
        fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
    ms_seq = timed(sequential)
    seq_phi = [p.clone() for p in ph]
    ms_bat = timed(batched)
    same = all(bool(torch.equal(a, c)) for a, c in zip(seq_phi, ph))
    b.close()
    for h in hs:
        h.close()
    by_size = {}
    for sp in specs:
        by_size[str(sp["levels"][-1])] = by_size.get(str(sp["levels"][-1]), 0) + sp["J"]
    return {"problems": len(specs), "particles": total, "particles_by_finest_inv_h": by_size,
            "sequential_ms": ms_seq, "batched_graph_ms": ms_bat,
            "sequential_evals_per_s": total / (ms_seq * 1e-3), "batched_evals_per_s": total / (ms_bat * 1e-3),
            "speedup": ms_seq / ms_bat, "identical_potentials": same}


def batched_sampler_measurement(native, wl, torch, dev, n_problems=64, max_inv_h=128, j_range=(500, 8000)):
    """The batched workload's samplers to their posteriors: n_problems independent MLS^2MC problems of
    uneven size (finest 1/h from {16, 32, 64, 128}, K from {16, 32, 64}, J log-uniform in j_range,
    5 pCN steps, mixed precision; problem p's sampler seed 300 + p), each run alone with smc_run, one
    after another, against all of them advanced together by the batched sampler (smc_batch_run: every
    problem's next update in shared launches). Data as in batched_measurement. Wall seconds on the
    host clock with the stream synchronised; whether every problem's path and particles agree."""
    specs = wl.batched_uneven(n_problems=n_problems, max_inv_h=max_inv_h, j_range=j_range)
    stream = torch.cuda.Stream(dev)
    s = stream.cuda_stream
    obs = wl.obs_grid(7)
    kws = []
    for p, sp in enumerate(specs):
        h0 = native.Handle(sp["levels"], sp["K"], obs, np.zeros(49), 1.0, corr_len=sp["corr_len"],
                           precision=native.SMC_MIXED, stream=s)
        G, _ = h0.eval_likelihood(len(sp["levels"]) - 1, wl.standard_normals((1, sp["K"]), sp["seed_true"]))
        h0.close()
        sigma = 0.01 * float(np.abs(G).max())
        y = G[0] + sigma * wl.standard_normals((49,), sp["seed_noise"])
        kws.append(dict(inv_h=list(sp["levels"]), K=sp["K"], obs_xy=obs, y=y, sigma=sigma, corr_len=sp["corr_len"],
                        J=sp["J"], n_mcmc=5, precision=native.SMC_MIXED, seed=300 + p, stream=s))

    def make(kw):
        kw = dict(kw)
        return native.Handle(kw.pop("inv_h"), kw.pop("K"), kw.pop("obs_xy"), kw.pop("y"), kw.pop("sigma"), **kw)

    seq = [make(kw) for kw in kws]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for h in seq:
        h.run()
    stream.synchronize()
    t_seq = time.perf_counter() - t0
    bat = [make(kw) for kw in kws]
    b = native.Batch(bat)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    steps = b.run()
    stream.synchronize()
    t_bat = time.perf_counter() - t0
    same_particles = [bool(np.array_equal(x.particles()[0], z.particles()[0])) for x, z in zip(seq, bat)]
    same_state = [x.state() == z.state() for x, z in zip(seq, bat)]
    same_path = [x.path() == z.path() for x, z in zip(seq, bat)]
    same = all(same_particles) and all(same_state) and all(same_path)
    differ = []
    for p, (x, z) in enumerate(zip(seq, bat)):
        if same_particles[p] and same_state[p] and same_path[p]:
            continue
        px, pz = x.path(), z.path()
        first = next((i for i, (a, c) in enumerate(zip(px, pz)) if a != c), min(len(px), len(pz)))
        fields = sorted(k for k in px[first] if first < len(px) and first < len(pz) and px[first][k] != pz[first][k]) \
            if first < min(len(px), len(pz)) else ["length"]
        differ.append({"problem": p, "levels": specs[p]["levels"], "K": specs[p]["K"], "J": specs[p]["J"],
                       "first_differing_update": first, "updates": [len(px), len(pz)], "fields": fields})
    updates = sum(h.state()["n_updates"] for h in bat)
    b.close()
    for h in seq + bat:
        h.close()
    by_size = {}
    for sp in specs:
        by_size[str(sp["levels"][-1])] = by_size.get(str(sp["levels"][-1]), 0) + 1
    return {"problems": len(specs), "particles": int(sum(sp["J"] for sp in specs)), "problems_by_finest_inv_h": by_size,
            "sequential_s": t_seq, "batched_s": t_bat, "speedup": t_seq / t_bat, "batched_steps": steps,
            "updates": updates, "identical_paths_and_particles": bool(same),
            "problems_with_identical": {"particles": int(sum(same_particles)), "state": int(sum(same_state)),
                                        "path": int(sum(same_path))}, "differing": differ}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-run", action="store_true", help="skip the seconds-to-posterior sampler run")
    ap.add_argument("--autotune", action="store_true", help="let the library's autotuner pick the block sizes")
    ap.add_argument("--large", action="store_true",
                    help="also run the large workload (1/16 .. 1/256, K = 128, J = 16384): the prescribed "
                         "pCN step against the adaptive step, plain and screened, with per-update diagnostics")
    ap.add_argument("--example-5-3-full", action="store_true",
                    help="also run Example 5.3 at the paper's size (1/16 .. 1/256, 320 KL terms)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_1709_09763_gb300 import build, native
    from paper_1709_09763_gb300 import workloads as wl

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    w = wl.WORKLOADS[WORKLOAD]
    d = load_data()
    obs = wl.obs_grid(w.obs_per_side)
    stream = torch.cuda.current_stream(dev)
    J, L, n_obs = w.J, len(w.inv_h), w.n_obs
    h = native.Handle(w.inv_h, w.K, obs, d["y"], d["sigma"], corr_len=w.corr_len, variance=w.variance, J=J,
                      J_tilde=w.J_tilde, n_mcmc=1, s_pcn=w.s_pcn, tau_star=w.tau_star,
                      precision=native.SMC_MIXED, seed=w.seed_sampler + 1000 * rank, stream=stream.cuda_stream)
    theta0 = wl.particles(J, w.K, 1000 + rank)
    if args.autotune:                   # block size per level, chosen by the library's autotuner
        tuned, _ = h.autotune(J)
    else:                               # the library's defaults (its fastest forms at this J)
        tuned = [h.block_size(l) for l in range(L)]
    h.set_particles(theta0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2
    # one step: on every level a tempering update (Phi of all particles, adaptive increment,
    # resampling, n_mcmc pCN sweeps) and, below the finest level, a bridging step to the next level
    # (Phi on both levels, adaptive zeta increment, resampling, n_mcmc pCN sweeps solving both levels
    # per proposal, Sec. 4.1): the sampler's two update kinds with the workload's 5 pCN steps
    n_mcmc_step = w.n_mcmc
    evals_level = [J * (1 + n_mcmc_step) + (2 * J * (1 + n_mcmc_step) if l < L - 1 else 0) for l in range(L)]
    evals_per_step = int(sum(evals_level))

    def step(ev=None):
        for l in range(L):
            if ev is not None:
                ev[l][0].record(stream)
            h.tempering_update(l, 0.0, n_mcmc_step)
            if l < L - 1:
                h.bridging_update(l, 1.0, 0.0, n_mcmc_step)
            if ev is not None:
                ev[l][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    h.get_timing()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    h.set_timing(True)
    lib = native.load()
    launches0 = lib.smc_kernel_launches()
    step_ms, level_ms = [], [[] for _ in range(L)]
    for _ in range(args.steps):
        flush.zero_()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(L)]
        step(ev)
        torch.cuda.synchronize(dev)
        for l in range(L):
            level_ms[l].append(ev[l][0].elapsed_time(ev[l][1]))
        step_ms.append(ev[0][0].elapsed_time(ev[L - 1][1]))
    torch.cuda.synchronize(dev)
    launches = lib.smc_kernel_launches() - launches0
    h.set_timing(False)
    kern_ms, kern_n = h.get_timing()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = float(np.mean(step_ms))

    # mean CG iterations of the finest-level solve on these particles (outside the timed region)
    th_now, _ = h.particles()
    tdev = torch.from_numpy(th_now).to(dev)
    Gd = torch.empty((J, n_obs), dtype=torch.float64, device=dev)
    Pd = torch.empty(J, dtype=torch.float64, device=dev)
    It = torch.empty(J, dtype=torch.int32, device=dev)
    h.eval_likelihood_device(L - 1, J, tdev.data_ptr(), Gd.data_ptr(), Pd.data_ptr(), It.data_ptr(),
                             stream.cuda_stream)
    it = It.cpu().numpy()
    if (it <= 0).any():
        raise RuntimeError("a forward solve did not converge")

    # e2e through the host-pointer C-ABI: particles in from pinned host memory, particles and
    # potentials out, every step
    th_host = torch.empty((J, w.K), dtype=torch.float64, pin_memory=True)
    th_host.numpy()[:] = theta0
    th_out = torch.empty((J, w.K), dtype=torch.float64, pin_memory=True)
    phi_out = torch.empty(J, dtype=torch.float64, pin_memory=True)
    ptr = lambda a: a.numpy().ctypes.data_as(native._dp)

    def e2e_step():
        h._check(lib.smc_set_particles(h._h, ptr(th_host)))
        step()
        h._check(lib.smc_get_particles(h._h, ptr(th_out), ptr(phi_out)))
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms.append(e0.elapsed_time(e1))
    e2e = float(np.mean(e2e_ms))
    # the step's evaluations only: smc_set_particles also evaluates Phi on the coarsest level (J cheap
    # solves), which the timed region includes but the count leaves out
    e2e_evals = evals_per_step

    # seconds to posterior: full MLS^2MC runs (n_mcmc = 5) of the workload from the prior, plain pCN and
    # delayed-acceptance pCN screened by the surrogate, R seeds each, outside the timed region
    run = None
    if not args.no_run:
        def one_run(wk, dk, inv_h, surrogate, seed, precision=native.SMC_MIXED, marginals=False, breakdown=False,
                    accept_target=0.0):
            ob = wl.obs_grid(wk.obs_per_side)
            hr = native.Handle(inv_h, wk.K, ob, dk["y"], dk["sigma"], corr_len=wk.corr_len, variance=wk.variance,
                               J=wk.J, J_tilde=wk.J_tilde, n_mcmc=wk.n_mcmc, s_pcn=wk.s_pcn,
                               tau_star=wk.tau_star, precision=precision, seed=seed,
                               stream=stream.cuda_stream, surrogate=surrogate, cov=wk.cov, source=wk.source,
                               proposal=wk.proposal, bc=wk.bc, tau_min=wk.tau_min, accept_target=accept_target)
            if breakdown:
                hr.set_timing(True)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hr.run()
            torch.cuda.synchronize(dev)
            secs = time.perf_counter() - t0
            st = hr.state()
            path = hr.path()
            m, v, lz = hr.posterior_moments()
            extra = {}
            if breakdown:
                # device time by part of the run (events on the handle's stream; a separate run from
                # the timed ones): forward solves per level, surrogate training and inference,
                # screening, increments and resampling, Markov moves, the gate's calibration
                sms, scnt = hr.get_timing()
                extra["breakdown_ms"] = {"solves_per_level": sms[:len(inv_h)].tolist(),
                                         "solve_launches_per_level": scnt[:len(inv_h)], **hr.get_phase_timing()}
                extra["breakdown_ms"]["wall_ms"] = secs * 1e3
                hr.set_timing(False)
            if marginals:
                # the leading three coefficients' particles (KS distances) and Phi of the posterior
                # mean on the finest level (Eq. RelMisfit), outside the timed region
                th_all = hr.particles()[0]
                extra["marginals"] = th_all[:, :3].copy()
                extra["unique_particles"] = int(np.unique(th_all, axis=0).shape[0])
                extra["accept_mean"] = float(np.mean([p["accept_rate"] for p in path])) if path else None
                extra["phi_at_mean"] = float(hr.eval_likelihood(len(inv_h) - 1, np.asarray(m)[None, :])[1][0])
            hr.close()
            rates = [p["da_stage1_rate"] for p in path if p["da_stage1_rate"] >= 0]
            return {"seconds": secs, "updates": st["n_updates"], "solves_per_level": st["evals"][:len(inv_h)],
                    "final_level": st["level"],
                    "log_evidence": lz, "mean": m, "var": v,
                    "stage1_pass_rate": float(np.mean(rates)) if rates else None, **extra}

        def fp64_solve_roofline(wk, dk, reps=5):
            """The FP64 solve of the single-level workload against the FP64 FMA issue peak: J
            particles on its level, the library's launch timing, the algorithm's FP64 operations
            (KL synthesis in the solve kernel, MG-PCG iterations, one residual check)."""
            hr = native.Handle(list(wk.inv_h), wk.K, wl.obs_grid(wk.obs_per_side), dk["y"], dk["sigma"],
                               corr_len=wk.corr_len, variance=wk.variance, J=wk.J, precision=native.SMC_FP64,
                               stream=stream.cuda_stream)
            th = torch.from_numpy(wl.particles(wk.J, wk.K, 31)).to(dev)
            Pp = torch.empty(wk.J, dtype=torch.float64, device=dev)
            Ii = torch.empty(wk.J, dtype=torch.int32, device=dev)
            hr.eval_likelihood_device(0, wk.J, th.data_ptr(), 0, Pp.data_ptr(), Ii.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize(dev)
            hr.get_timing()
            hr.set_timing(True)
            for _ in range(reps):
                flush.zero_()
                hr.eval_likelihood_device(0, wk.J, th.data_ptr(), 0, Pp.data_ptr(), Ii.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize(dev)
            km, kn = hr.get_timing()
            hr.close()
            its = Ii.cpu().numpy()
            launch_ms = km[0] / max(kn[0], 1)
            N = wk.inv_h[0]
            fl = algorithmic_flops_per_eval(N, wk.K, float(its.mean()), 1.0, synthesis=True)
            peaks, _ = measured_peaks()
            peak = 152 * 2 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            ach = fl * wk.J / (launch_ms * 1e-3) / 1e12
            return {"kernel": f"fem_eval_kernel<double,{N}>",
                    "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "launch_ms": launch_ms, "evals_per_s": wk.J / (launch_ms * 1e-3),
                    "mean_cg_iters": float(its.mean()), "flops_per_eval": fl,
                    "peak_source": "FP64 FMA issue: 152 SMs x 2 FMA per clock x 2 flops x sm_max_mhz "
                                   "(the 1.25 TFLOP/s FP64 figure of this part)"}

        def compare(wk, dk, inv_h, R=3, breakdown=False, accept_target=0.0):
            """Plain and surrogate-screened MLS^2MC, R seeds each (the same seeds for both arms): wall
            seconds to the posterior, the posterior means' agreement (largest |z| over the K
            coordinates of the two arms' replicate means) and the speed-up of the medians with a 95 %
            bootstrap interval (runs resampled within each arm, 2000 draws, fixed seed)."""
            res = {}
            for name, sur in (("plain", 0), ("surrogate", 1)):
                runs = [one_run(wk, dk, inv_h, sur, wk.seed_sampler + 1000 * rank + 17 * r,
                                accept_target=accept_target) for r in range(R)]
                res[name] = {"seconds_median": float(np.median([x["seconds"] for x in runs])),
                             "seconds": [x["seconds"] for x in runs],
                             "solves_per_level_mean": np.mean([x["solves_per_level"] for x in runs], axis=0).tolist(),
                             "updates": [x["updates"] for x in runs],
                             "log_evidence": [x["log_evidence"] for x in runs],
                             "stage1_pass_rate": runs[0]["stage1_pass_rate"],
                             "_means": np.array([x["mean"] for x in runs])}
                if breakdown:
                    res[name]["breakdown_ms"] = one_run(wk, dk, inv_h, sur, wk.seed_sampler + 1000 * rank,
                                                        breakdown=True, accept_target=accept_target)["breakdown_ms"]
            a, b = res["plain"].pop("_means"), res["surrogate"].pop("_means")
            se = np.sqrt(a.var(axis=0, ddof=1) / R + b.var(axis=0, ddof=1) / R)
            z = np.abs(a.mean(0) - b.mean(0)) / np.where(se > 0, se, np.inf)
            tp, ts = np.array(res["plain"]["seconds"]), np.array(res["surrogate"]["seconds"])
            rng_b = np.random.default_rng(12345)
            boot = [np.median(rng_b.choice(tp, R)) / np.median(rng_b.choice(ts, R)) for _ in range(2000)]
            return {"workload": wk.name, "levels_inv_h": list(inv_h), "K": wk.K, "J": wk.J, "n_mcmc": wk.n_mcmc,
                    "s_pcn": wk.s_pcn, "accept_target": accept_target,
                    "replicates": R, "plain": res["plain"], "surrogate": res["surrogate"],
                    "speedup_surrogate_vs_plain": res["plain"]["seconds_median"] / res["surrogate"]["seconds_median"],
                    "speedup_ci95": [float(np.percentile(boot, 2.5)), float(np.percentile(boot, 97.5))],
                    "posterior_mean_diff_over_se_max": float(np.max(z))}
        # MLS^2MC on the workload's hierarchy, single-level SMC on its finest level (Example
        # example_SMC, the paper's reference sampler), and the surrogate workload (5 levels to 1/128,
        # K = 64, J = 8000, 10 pCN steps): plain pCN vs surrogate-screened pCN
        wda = wl.WORKLOADS["da_mixed_h8_128"]
        dda = load_data(wda.name)
        run = {"mls2mc": compare(w, d, tuple(w.inv_h)), "smc_finest": compare(w, d, (w.inv_h[-1],), R=6),
               "mls2mc_surrogate_workload": compare(wda, dda, tuple(wda.inv_h), R=8, breakdown=True),
               "mls2mc_surrogate_workload_adaptive_step": compare(wda, dda, tuple(wda.inv_h), R=8, breakdown=True,
                                                                  accept_target=0.25),
               # the same workload with the covariance-shaped random walk (first step 2.38 / sqrt(K), adaptive)
               "mls2mc_surrogate_workload_covariance_walk": compare(
                   dataclasses.replace(wda, proposal="rwm_cov", s_pcn=2.38 / math.sqrt(wda.K)), dda,
                   tuple(wda.inv_h), R=8, breakdown=True, accept_target=0.25)}

        def paper_example(name, R=3, J_sweep=()):
            """The paper's examples (Matern prior, one random-walk step per update; 5.1/5.2: nine
            sources, 5.3: the flow cell under the scheme u'): MLS^2MC on the hierarchy against
            single-level SMC on its finest level, R seeded runs each; cost in the paper's unit
            sum_l evals_l 4^(l - L) (one finest-level solve = 1). Accuracy as in Sec. 5.1: RelErr
            and RelMisfit of each run's posterior mean, KS distances of the theta_1..theta_3
            marginals between the runs of the two samplers and within single-level SMC (the base
            scatter), RelErrEvid against the geometric mean of the single-level SMC evidences.
            J_sweep: the same comparison (R // 2 runs each) at smaller J, for cost against accuracy."""
            from paper_1709_09763_gb300 import metrics
            wk, dk = wl.WORKLOADS[name], load_data(name)
            res = {"workload": name, "levels_inv_h": list(wk.inv_h), "K": wk.K, "J": wk.J, "sigma": dk["sigma"],
                   "tau_star": wk.tau_star, "proposal": wk.proposal, "replicates": R}
            hk = native.Handle([wk.inv_h[0]], wk.K, wl.obs_grid(wk.obs_per_side), dk["y"], dk["sigma"],
                               corr_len=wk.corr_len, precision=native.SMC_MIXED, cov=wk.cov, source=wk.source)
            lam = hk.kl_table(0, wk.inv_h[0])[1]
            hk.close()
            th_true = np.array(dk["theta_true"])

            def arm(wj, inv_h, n):
                runs = [one_run(wj, dk, inv_h, 0, wj.seed_sampler + 1000 * rank + 17 * r, marginals=True)
                        for r in range(n)]
                L = len(inv_h)
                cost = [float(sum(e * 4.0 ** (l - (L - 1)) for l, e in enumerate(x["solves_per_level"]))) for x in runs]
                return runs, {"seconds_median": float(np.median([x["seconds"] for x in runs])),
                              "seconds": [x["seconds"] for x in runs],
                              "solves_per_level_mean": np.mean([x["solves_per_level"] for x in runs], axis=0).tolist(),
                              "cost_finest_solves_mean": float(np.mean(cost)),
                              "updates": [x["updates"] for x in runs],
                              "log_evidence": [x["log_evidence"] for x in runs],
                              "rel_err_posterior_mean": [metrics.rel_err(x["mean"], th_true, lam) for x in runs],
                              "rel_misfit_posterior_mean": [metrics.rel_misfit(x["phi_at_mean"], dk["y"], dk["sigma"])
                                                            for x in runs],
                              "final_level_inv_h": [inv_h[x["final_level"]] for x in runs],
                              "unique_particles_median": float(np.median([x["unique_particles"] for x in runs])),
                              "accept_rate_mean": float(np.mean([x["accept_mean"] for x in runs]))}

            def accuracy(ml_runs, sl_runs):
                ref = metrics.log_z_ref([x["log_evidence"] for x in sl_runs])
                ks_ml, ks_ml_sd, n_ml = metrics.pairwise_ks([x["marginals"] for x in ml_runs],
                                                             [x["marginals"] for x in sl_runs])
                ks_sl, ks_sl_sd, n_sl = metrics.pairwise_ks([x["marginals"] for x in sl_runs])
                ree = lambda rs: metrics.rel_err_evid([x["log_evidence"] for x in rs], ref)
                return {"ks_mls2mc_vs_smc_mean": ks_ml.tolist(), "ks_mls2mc_vs_smc_sd": ks_ml_sd.tolist(),
                        "ks_pairs": n_ml, "ks_smc_vs_smc_mean": ks_sl.tolist(), "ks_smc_vs_smc_sd": ks_sl_sd.tolist(),
                        "log_z_ref": ref, "rel_err_evid_mls2mc_mean": float(np.mean(ree(ml_runs))),
                        "rel_err_evid_smc_mean": float(np.mean(ree(sl_runs)))}

            ml_runs, res["mls2mc"] = arm(wk, tuple(wk.inv_h), R)
            sl_runs, res["smc_finest"] = arm(wk, (wk.inv_h[-1],), R)
            res["speedup_mls2mc_vs_smc"] = res["smc_finest"]["seconds_median"] / res["mls2mc"]["seconds_median"]
            res["cost_ratio_smc_over_mls2mc"] = (res["smc_finest"]["cost_finest_solves_mean"] /
                                                 res["mls2mc"]["cost_finest_solves_mean"])
            if R >= 2:
                res["accuracy"] = accuracy(ml_runs, sl_runs)
            if J_sweep:
                # cost against accuracy: finest-level solve equivalents and seconds vs RelErr per J
                table = []
                for J in J_sweep:
                    wj = dataclasses.replace(wk, J=J)
                    n = max(2, R // 2)
                    mr, ms = arm(wj, tuple(wk.inv_h), n)
                    sr, ss = arm(wj, (wk.inv_h[-1],), n)
                    for label, st in (("mls2mc", ms), ("smc_finest", ss)):
                        table.append({"J": J, "sampler": label, "runs": n,
                                      "cost_finest_solves": st["cost_finest_solves_mean"],
                                      "seconds_median": st["seconds_median"],
                                      "rel_err_mean": float(np.mean(st["rel_err_posterior_mean"])),
                                      "rel_err_sd": float(np.std(st["rel_err_posterior_mean"])),
                                      "rel_misfit_mean": float(np.mean(st["rel_misfit_posterior_mean"]))})
                res["cost_vs_accuracy"] = table
            return res
        def large_study(R=4):
            """The large workload (5 levels 1/16 .. 1/256, K = 128, 144 interpolated observations, J =
            16384, 10 Markov steps): pCN with the prescribed step s = 0.2 against pCN with the adaptive
            step (accept_target 0.25) and the covariance-shaped random walk (first step 2.38 / sqrt(K),
            adaptive), plain and screened; per update the acceptance rate, the distinct ancestors its
            resampling kept and the step; across replicates the spread of the posterior means and of
            log Z, and the largest |z| between the arms' replicate means."""
            wk, dk = wl.WORKLOADS["large_mixed_h16_256"], load_data("large_mixed_h16_256")
            ob = wl.obs_grid(wk.obs_per_side)
            out = {"workload": wk.name, "levels_inv_h": list(wk.inv_h), "K": wk.K, "J": wk.J, "n_mcmc": wk.n_mcmc,
                   "replicates": R}
            means = {}
            s_cov = 2.38 / math.sqrt(wk.K)
            for label, sur, target, prop, s0 in (("prescribed_step", 0, 0.0, "pcn", wk.s_pcn),
                                                 ("adaptive_step", 0, 0.25, "pcn", wk.s_pcn),
                                                 ("adaptive_step_screened", 1, 0.25, "pcn", wk.s_pcn),
                                                 ("covariance_walk", 0, 0.25, "rwm_cov", s_cov),
                                                 ("covariance_walk_screened", 1, 0.25, "rwm_cov", s_cov)):
                runs = []
                for r in range(R):
                    hr = native.Handle(list(wk.inv_h), wk.K, ob, dk["y"], dk["sigma"], corr_len=wk.corr_len,
                                       J=wk.J, J_tilde=wk.J_tilde, n_mcmc=wk.n_mcmc, s_pcn=s0,
                                       tau_star=wk.tau_star, precision=native.SMC_MIXED,
                                       seed=wk.seed_sampler + 1000 * rank + 17 * r, stream=stream.cuda_stream,
                                       surrogate=sur, accept_target=target, proposal=prop)
                    torch.cuda.synchronize(dev)
                    t0 = time.perf_counter()
                    hr.run()
                    torch.cuda.synchronize(dev)
                    secs = time.perf_counter() - t0
                    path = hr.path()
                    m, v, lz = hr.posterior_moments()
                    st = hr.state()
                    hr.close()
                    runs.append({"seconds": secs, "updates": len(path), "log_z": lz, "mean": np.asarray(m),
                                 "solves_per_level": st["evals"][:len(wk.inv_h)],
                                 "accept": [round(p["accept_rate"], 4) for p in path],
                                 "n_unique": [p["n_unique"] for p in path],
                                 "step": [round(p["step"], 5) for p in path],
                                 "kind_level": [f'{p["kind"]}{p["level"]}' for p in path]})
                M = np.array([x["mean"] for x in runs])
                means[label] = M
                out[label] = {"seconds": [x["seconds"] for x in runs],
                              "seconds_median": float(np.median([x["seconds"] for x in runs])),
                              "updates": [x["updates"] for x in runs], "log_z": [x["log_z"] for x in runs],
                              "solves_per_level_mean": np.mean([x["solves_per_level"] for x in runs], axis=0).tolist(),
                              "replicate_sd_of_mean_max": float(M.std(axis=0, ddof=1).max()),
                              "replicate_sd_of_mean_median": float(np.median(M.std(axis=0, ddof=1))),
                              "log_z_sd": float(np.std([x["log_z"] for x in runs], ddof=1)),
                              "first_run": {k: runs[0][k] for k in ("accept", "n_unique", "step", "kind_level")}}

            def zmax(a, b):
                se = np.sqrt(a.var(axis=0, ddof=1) / len(a) + b.var(axis=0, ddof=1) / len(b))
                return float(np.max(np.abs(a.mean(0) - b.mean(0)) / np.where(se > 0, se, np.inf)))

            def welch(a, b, fwer=0.05):
                """Largest Welch t over the K coordinates of two arms' replicate means, its coordinate's
                degrees of freedom, and the critical value of a family-wise false-alarm rate fwer
                (Bonferroni over K, two-sided) at those degrees of freedom."""
                from scipy.stats import t as student_t
                va, vb = a.var(axis=0, ddof=1) / len(a), b.var(axis=0, ddof=1) / len(b)
                tv = np.abs(a.mean(0) - b.mean(0)) / np.sqrt(va + vb)
                k = int(np.argmax(tv))
                dof = (va[k] + vb[k]) ** 2 / (va[k] ** 2 / (len(a) - 1) + vb[k] ** 2 / (len(b) - 1))
                crit = float(student_t.ppf(1.0 - fwer / (2 * a.shape[1]), dof))
                return {"t_max": float(tv[k]), "dof": float(dof), "critical": crit, "agree": bool(tv[k] < crit)}
            out["z_max_adaptive_vs_prescribed"] = zmax(means["adaptive_step"], means["prescribed_step"])
            out["z_max_screened_vs_plain_adaptive"] = zmax(means["adaptive_step_screened"], means["adaptive_step"])
            out["speedup_screened_vs_plain_adaptive"] = (out["adaptive_step"]["seconds_median"] /
                                                        out["adaptive_step_screened"]["seconds_median"])
            out["z_max_covariance_walk_screened_vs_plain"] = zmax(means["covariance_walk_screened"],
                                                                  means["covariance_walk"])
            out["z_max_covariance_walk_vs_adaptive_pcn"] = zmax(means["covariance_walk"], means["adaptive_step"])
            out["speedup_covariance_walk_screened_vs_plain"] = (out["covariance_walk"]["seconds_median"] /
                                                               out["covariance_walk_screened"]["seconds_median"])
            out["welch_covariance_walk_screened_vs_plain"] = welch(means["covariance_walk_screened"],
                                                                   means["covariance_walk"])
            out["welch_adaptive_pcn_screened_vs_plain"] = welch(means["adaptive_step_screened"], means["adaptive_step"])
            out["welch_covariance_walk_vs_adaptive_pcn"] = welch(means["covariance_walk"], means["adaptive_step"])
            return out

        # single-level SMC on the FP64 path (h = 1/16, K = 16, J = 1000, 5 pCN steps)
        wf, dfp = wl.WORKLOADS["smc_fp64_h16"], load_data("smc_fp64_h16")
        fr = [one_run(wf, dfp, tuple(wf.inv_h), 0, wf.seed_sampler + 17 * r, native.SMC_FP64) for r in range(3)]
        run["smc_fp64_h16"] = {"workload": wf.name, "levels_inv_h": list(wf.inv_h), "K": wf.K, "J": wf.J,
                               "n_mcmc": wf.n_mcmc, "precision": "fp64",
                               "seconds_median": float(np.median([x["seconds"] for x in fr])),
                               "seconds": [x["seconds"] for x in fr],
                               "solves_mean": float(np.mean([x["solves_per_level"][0] for x in fr])),
                               "solves_per_s": float(np.mean([x["solves_per_level"][0] / x["seconds"] for x in fr])),
                               "updates": [x["updates"] for x in fr],
                               "log_evidence": [x["log_evidence"] for x in fr],
                               "roofline": fp64_solve_roofline(wf, dfp)}
        run["paper_example_5_1"] = paper_example("example_5_1", R=12, J_sweep=(625, 1250))
        run["paper_example_5_2"] = paper_example("example_5_2", R=12, J_sweep=(625, 1250))
        # Example 5.3, the flow cell, at reduced size (levels 1/16 .. 1/64, 64 KL terms), scheme u'
        run["paper_example_5_3"] = paper_example("example_5_3")
        if args.example_5_3_full:   # the paper's size: 1/16 .. 1/256, 320 KL terms
            run["paper_example_5_3_full"] = paper_example("example_5_3_full")
        if args.large:
            run["large_workload"] = large_study()

    batched = None if args.no_run else batched_measurement(native, wl, torch, dev)
    batched_run = None if args.no_run else batched_sampler_measurement(native, wl, torch, dev)
    # many small problems' samplers: each sequential run fills a fraction of the GPU
    batched_run_small = None if args.no_run else batched_sampler_measurement(native, wl, torch, dev,
                                                                             n_problems=256, max_inv_h=64,
                                                                             j_range=(64, 512))
    # many small problems: each per-problem launch fills a fraction of the GPU
    batched_small = None if args.no_run else batched_measurement(native, wl, torch, dev, n_problems=256,
                                                                 max_inv_h=64, j_range=(16, 256))

    t = reduce_max_over_ranks([ms, e2e] + [float(np.mean(x)) for x in level_ms], dist if world > 1 else None, dev)
    ms, e2e = t[0], t[1]
    lvl_ms = t[2:]
    if rank == 0:
        peaks, src = measured_peaks()
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12      # TFLOP/s, FMA = 2 flops
        mean_it = float(it.mean())
        kl = L - 1
        launch_ms = kern_ms[kl] / max(kern_n[kl], 1)
        per_particle = FEM64_DRAM_BYTES_PER_PARTICLE.get(tuned[-1]) if w.inv_h[-1] == 64 else None
        traffic = per_particle * J if per_particle is not None else None
        flops = algorithmic_flops_per_eval(w.inv_h[-1], w.K, mean_it, 2.0) * J
        achieved = flops / (launch_ms * 1e-3) / 1e12
        smem_tbs = algorithmic_smem_bytes_per_eval(w.inv_h[-1], mean_it, 2.0) * J / (launch_ms * 1e-3) / 1e12
        smem_peak = 152 * 128 * sm_mhz * 1e6 / 1e12           # TB/s, one 128-byte wavefront per SM cycle
        total_evals = evals_per_step * world
        line = {
            "metric": "likelihood evals/s per mesh level", "value": job_throughput(evals_per_step, world, ms),
            "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels_inv_h": list(w.inv_h), "K": w.K, "n_obs": n_obs, "J": J,
                       "precision": "mixed", "step": "per level: a tempering update (Phi on all particles, "
                       "adaptive increment, systematic resampling, 5 pCN sweeps) and, below the finest level, a "
                       "bridging step to the next level (Phi on both levels, adaptive zeta increment, "
                       "resampling, 5 pCN sweeps solving both levels per proposal)",
                       "evals_per_step": evals_per_step, "l2": "flushed between steps (256 MB write)",
                       "threads_per_particle": dict(zip([str(N) for N in w.inv_h], tuned)),
                       "parallelism": f"replicas x{world}"},
            "per_level": {str(N): {"evals_per_s": evals_level[l] * world / (lm * 1e-3), "update_ms": lm,
                                   "evals": evals_level[l],
                                   "solve_launch_ms": kern_ms[l] / max(kern_n[l], 1),
                                   "solve_evals_per_s": J / (kern_ms[l] / max(kern_n[l], 1) * 1e-3),
                                   "solve_kernel": solve_kernel_name(N, tuned[l]),
                                   # shared-memory roofline of the level's solve (mean CG iterations
                                   # of the finest level stand in for every level: 10-12 measured)
                                   "smem_frac": algorithmic_smem_bytes_per_eval(N, mean_it, 2.0) * J /
                                   (kern_ms[l] / max(kern_n[l], 1) * 1e-3) / 1e12 / smem_peak}
                          for l, (N, lm) in enumerate(zip(w.inv_h, lvl_ms))},
            "roofline": {"kernel": solve_kernel_name(w.inv_h[-1], tuned[-1]), "bound": "alu",
                         "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak,
                         "traffic": traffic,
                         "launch_ms": launch_ms,
                         "launches": kern_n[kl], "mean_cg_iters": mean_it,
                         "peak_source": f"FP32 FMA issue rate: 152 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz "
                                        f"(sm_max_mhz {src})"},
            # the bound that holds the solve: the shared-memory pipe (the FP32 issue roofline above
            # is the contract's "alu" figure; the solve runs on chip, far from both HBM and ALU)
            "roofline_smem": {"kernel": solve_kernel_name(w.inv_h[-1], tuned[-1]), "bound": "smem",
                              "achieved": smem_tbs, "peak": smem_peak, "unit": "TB/s",
                              "frac": smem_tbs / smem_peak,
                              "peak_source": f"152 SMs x 128 B per cycle x {sm_mhz:.0f} MHz"},
            "e2e": {"value": job_throughput(e2e_evals, world, e2e), "unit": "evals/s",
                    "h2d_bytes_per_step": J * w.K * 8, "d2h_bytes_per_step": J * (w.K + 1) * 8},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if run is not None:
            line["seconds_to_posterior"] = run
        if batched is not None:
            line["batched_uneven"] = batched
        if batched_small is not None:
            line["batched_small_problems"] = batched_small
        if batched_run is not None:
            line["batched_sampler_to_posterior"] = batched_run
        if batched_run_small is not None:
            line["batched_sampler_small_problems_to_posterior"] = batched_run_small
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
