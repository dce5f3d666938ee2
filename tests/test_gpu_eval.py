"""GPU parity of the likelihood path G_l(theta), Phi_l(theta) against the FP64 oracle.

Tolerances: per-particle observation vectors to 1e-10 relative (max-norm) on the
FP64 path, 1e-6 on the mixed path; Phi to the bound those G tolerances imply
through Phi = 1/2 |y - G|^2 / sigma^2 (the residual y - G cancels digits of G).
"""
import json
import os

import numpy as np
import pytest

from oracle import forward as ofwd
from oracle import kl as okl
from paper_1709_09763_gb300 import native
from paper_1709_09763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _data(name):
    with open(os.path.join(GOLD, f"data_{name}.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _oracle(N, w, theta, obs, y, sigma):
    lv = ofwd.Level(N, w.corr_len, w.variance, w.K, obs)
    G = lv.G_batch(theta)
    return G, ofwd.potential(G, y, sigma)


def _rel(a, b):
    return np.max(np.abs(a - b), axis=-1) / np.max(np.abs(b), axis=-1)


def _phi_ok(Phi, Phir, Gr, sigma, tol):
    """Phi tolerance implied by a max-norm relative tolerance `tol` on G:
    |dPhi| <= |y - G|_2 |dG|_2 / sigma^2 + |dG|_2^2 / (2 sigma^2), |y - G|_2 = sigma sqrt(2 Phi),
    |dG|_2 <= tol * max|G| * sqrt(n_obs)."""
    dG = tol * np.max(np.abs(Gr), axis=-1) * np.sqrt(Gr.shape[-1])
    bound = np.sqrt(2 * Phir) * dG / sigma + 0.5 * (dG / sigma) ** 2
    return np.all(np.abs(Phi - Phir) <= bound)


def test_kl_table_matches_oracle():
    w = wl.WORKLOADS["mls2mc_mixed_h8_64"]
    d = _data(w.name)
    h = native.Handle(w.inv_h, w.K, wl.obs_grid(7), d["y"], d["sigma"], corr_len=w.corr_len,
                      precision=native.SMC_MIXED)
    for l, N in enumerate(w.inv_h):
        psi, lam = h.kl_table(l, N)
        ref = okl.kl_table(N, w.corr_len, 1.0, w.K)
        assert np.abs(psi - ref).max() < 1e-12
        assert np.allclose(lam, [p[0] for p in okl.kl_pairs(w.corr_len, 1.0, w.K)], rtol=1e-13)


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_fp64_path_parity(N):
    w = wl.WORKLOADS["smc_fp64_h16"]
    d = _data(w.name)
    obs = wl.obs_grid(7)
    theta = wl.particles(37, w.K, 100 + N)           # 37: not a multiple of a warp
    h = native.Handle([N], w.K, obs, d["y"], d["sigma"], corr_len=w.corr_len, precision=native.SMC_FP64,
                      rtol=1e-13)
    G, Phi = h.eval_likelihood(0, theta)
    Gr, Phir = _oracle(N, w, theta, obs, np.array(d["y"]), d["sigma"])
    assert _rel(G, Gr).max() < 1e-10
    assert _phi_ok(Phi, Phir, Gr, d["sigma"], 1e-10)


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_mixed_path_parity(N):
    w = wl.WORKLOADS["mls2mc_mixed_h8_64"]
    d = _data(w.name)
    obs = wl.obs_grid(7)
    theta = wl.particles(23 if N == 64 else 41, w.K, 200 + N)
    h = native.Handle([N], w.K, obs, d["y"], d["sigma"], corr_len=w.corr_len, precision=native.SMC_MIXED)
    G, Phi = h.eval_likelihood(0, theta)
    Gr, Phir = _oracle(N, w, theta, obs, np.array(d["y"]), d["sigma"])
    assert _rel(G, Gr).max() < 1e-6
    assert _phi_ok(Phi, Phir, Gr, d["sigma"], 1e-6)


def test_interpolated_observations_and_small_K():
    """12 x 12 points at (i/13, j/13) are not mesh nodes: P1 barycentric interpolation; K = 1."""
    obs = wl.obs_grid(12)
    rng = np.random.default_rng(7)
    for K, prec, tol in ((1, native.SMC_FP64, 1e-10), (5, native.SMC_MIXED, 1e-6)):
        w = wl.Workload("t", (16,), 64, K, 0.2, 12, 0, 0)
        y = rng.normal(0, 0.01, 144)
        theta = wl.particles(9, K, 5)
        h = native.Handle([16], K, obs, y, 0.01, corr_len=0.2, precision=prec)
        G, Phi = h.eval_likelihood(0, theta)
        Gr, Phir = _oracle(16, w, theta, obs, y, 0.01)
        assert _rel(G, Gr).max() < tol


def test_empty_and_single_batches():
    w = wl.WORKLOADS["smc_fp64_h16"]
    d = _data(w.name)
    h = native.Handle([16], w.K, wl.obs_grid(7), d["y"], d["sigma"], corr_len=w.corr_len)
    G, Phi = h.eval_likelihood(0, np.zeros((0, w.K)))
    assert G.shape == (0, 49) and Phi.shape == (0,)
    theta = np.zeros((1, w.K))                        # kappa == 1: the torsion problem
    G, Phi = h.eval_likelihood(0, theta)
    Gr, _ = _oracle(16, w, theta, wl.obs_grid(7), np.array(d["y"]), d["sigma"])
    assert _rel(G, Gr).max() < 1e-10


def test_full_size_sampled_parity():
    """The benchmark's launch: J = 4000 particles on the 1/64 level (mixed); 6 sampled particles vs oracle."""
    import torch
    w = wl.WORKLOADS["mls2mc_mixed_h8_64"]
    d = _data(w.name)
    h = native.Handle(w.inv_h, w.K, wl.obs_grid(7), d["y"], d["sigma"], corr_len=w.corr_len,
                      precision=native.SMC_MIXED)
    theta = wl.particles(w.J, w.K, 4242)
    th = torch.from_numpy(theta).cuda()
    G = torch.empty((w.J, 49), dtype=torch.float64, device="cuda")
    Phi = torch.empty(w.J, dtype=torch.float64, device="cuda")
    it = torch.empty(w.J, dtype=torch.int32, device="cuda")
    h.eval_likelihood_device(3, w.J, th.data_ptr(), G.data_ptr(), Phi.data_ptr(), it.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(it.min()) > 0
    idx = np.array([0, 1, 777, 2048, 3998, 3999])
    Gr, Phir = _oracle(64, w, theta[idx], wl.obs_grid(7), np.array(d["y"]), d["sigma"])
    assert _rel(G.cpu().numpy()[idx], Gr).max() < 1e-6
    Phi = Phi.cpu().numpy()
    assert np.all(np.isfinite(Phi))
    assert _phi_ok(Phi[idx], Phir, Gr, d["sigma"], 1e-6)


@pytest.mark.parametrize("prec", [native.SMC_MIXED, native.SMC_FP64])
def test_every_block_size_and_autotuner(prec):
    """Each compiled threads-per-particle variant gives the oracle's G; the autotuner picks one of them."""
    w = wl.WORKLOADS["mls2mc_mixed_h8_64"]
    d = _data(w.name)
    obs = wl.obs_grid(7)
    levels = [8, 16, 32, 64] if prec == native.SMC_MIXED else [8, 16, 32]
    tol = 1e-6 if prec == native.SMC_MIXED else 1e-10
    h = native.Handle(levels, w.K, obs, d["y"], d["sigma"], corr_len=w.corr_len, precision=prec)
    sizes = {8: [32, 64], 16: [128, 64], 32: [256, 512, -256], 64: [512, 1024, -512]} if prec == native.SMC_MIXED else \
        {8: [64], 16: [128, 256], 32: [256, 512]}
    theta = wl.particles(9, w.K, 31)
    for l, N in enumerate(levels):
        Gr, _ = _oracle(N, w, theta, obs, np.array(d["y"]), d["sigma"])
        for T in sizes[N]:
            h.set_block_size(l, T)
            assert h.block_size(l) == T
            G, _ = h.eval_likelihood(l, theta)
            assert _rel(G, Gr).max() < tol, (N, T)
        h.set_block_size(l, 0)
        default = {32: -256, 64: -512}.get(N, sizes[N][0]) if prec == native.SMC_MIXED else sizes[N][0]
        assert h.block_size(l) == default, (N, h.block_size(l))
    with pytest.raises(native.SmcError):
        h.set_block_size(0, 96)
    with pytest.raises(native.SmcError):   # no compact form at 1/8, none with 128 threads at 1/32
        h.set_block_size(0, -32)
    if prec == native.SMC_MIXED:
        with pytest.raises(native.SmcError):
            h.set_block_size(2, -128)
    chosen, ms = h.autotune(256)
    assert all(c in sizes[N] for c, N in zip(chosen, levels)) and all(m > 0 for m in ms)
    for l in range(len(levels)):
        h.set_block_size(l, 0)


@pytest.mark.parametrize("N,n,B", [(128, 5, 1024), (128, 5, -1024), (128, 1, -1024), (256, 2, 0)])
def test_large_levels_parity(N, n, B):
    """1/h = 128 in both forms (1024: fine level in device memory; -1024: fine level on chip across the
    two CTAs of a cluster, also with a single particle) and 1/256: mixed-path G within 1e-6 of the
    oracle."""
    w = wl.WORKLOADS["mls2mc_mixed_h8_64"]
    d = _data(w.name)
    obs = wl.obs_grid(7)
    theta = wl.particles(n, w.K, 300 + N)
    h = native.Handle([N], w.K, obs, d["y"], d["sigma"], corr_len=w.corr_len, precision=native.SMC_MIXED)
    if B:
        h.set_block_size(0, B)
        assert h.block_size(0) == B
    G, Phi = h.eval_likelihood(0, theta)
    h.set_block_size(0, 0)
    Gr, Phir = _oracle(N, w, theta, obs, np.array(d["y"]), d["sigma"])
    assert _rel(G, Gr).max() < 1e-6
    assert _phi_ok(Phi, Phir, Gr, d["sigma"], 1e-6)


@pytest.mark.parametrize("N,K,corr,nobs,n", [(128, 64, 0.1, 7, 3), (256, 128, 0.05, 12, 2)])
def test_large_level_workload_shapes(N, K, corr, nobs, n):
    """The surrogate workload's finest level (1/128, K = 64) and the large workload's (1/256,
    K = 128, correlation length 0.05, 12 x 12 observations interpolated at (i/13, j/13)): mixed-path
    G within 1e-6 of the oracle."""
    obs = wl.obs_grid(nobs)
    theta = wl.particles(n, K, 900 + N)
    y = np.zeros(obs.shape[0])
    h = native.Handle([N], K, obs, y, 1.0, corr_len=corr, precision=native.SMC_MIXED)
    G, _ = h.eval_likelihood(0, theta)
    Gr = ofwd.Level(N, corr, 1.0, K, obs).G_batch(theta)
    assert _rel(G, Gr).max() < 1e-6, _rel(G, Gr)


@pytest.mark.parametrize("name", ["da_mixed_h8_128", "large_mixed_h16_256"])
def test_full_size_sampled_parity_large_workloads(name):
    """The finest-level launch of the surrogate workload (J = 8000 on 1/128, K = 64) and of the large
    workload (J = 16384 on 1/256, K = 128, 12 x 12 interpolated observations): every solve
    converges, sampled particles (first, last, inner) match the oracle within 1e-6."""
    import torch
    w = wl.WORKLOADS[name]
    d = _data(w.name)
    obs = wl.obs_grid(w.obs_per_side)
    h = native.Handle(w.inv_h, w.K, obs, d["y"], d["sigma"], corr_len=w.corr_len, precision=native.SMC_MIXED)
    theta = wl.particles(w.J, w.K, 5151)
    th = torch.from_numpy(theta).cuda()
    G = torch.empty((w.J, w.n_obs), dtype=torch.float64, device="cuda")
    Phi = torch.empty(w.J, dtype=torch.float64, device="cuda")
    it = torch.empty(w.J, dtype=torch.int32, device="cuda")
    L = len(w.inv_h) - 1
    h.eval_likelihood_device(L, w.J, th.data_ptr(), G.data_ptr(), Phi.data_ptr(), it.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(it.min()) > 0
    idx = np.array([0, 1, w.J // 3, w.J - 1])
    Gr, Phir = _oracle(w.inv_h[-1], w, theta[idx], obs, np.array(d["y"]), d["sigma"])
    assert _rel(G.cpu().numpy()[idx], Gr).max() < 1e-6
    assert _phi_ok(Phi.cpu().numpy()[idx], Phir, Gr, d["sigma"], 1e-6)


@pytest.mark.parametrize("K,J", [(32, 4000), (64, 8000)])
def test_cluster_form_agrees_with_device_memory_form(K, J):
    """1/128 at the surrogate workload's launch size (K = 64, J = 8000) and at J = 4000: the two-CTA
    form (the default) and the device-memory form run the same algorithm except for the rounding of
    the fine level's smoother diagonal, so every solve converges in both, the iteration counts
    differ by at most one and the observations agree far inside the 1e-6 parity bar."""
    import torch
    obs = wl.obs_grid(7)
    h = native.Handle([128], K, obs, np.zeros(49), 1.0, corr_len=0.1, precision=native.SMC_MIXED)
    assert h.block_size(0) == -1024
    theta = torch.from_numpy(wl.particles(J, K, 5151)).cuda()
    out = {}
    for B in (1024, -1024):
        h.set_block_size(0, B)
        G = torch.empty((J, 49), dtype=torch.float64, device="cuda")
        Phi = torch.empty(J, dtype=torch.float64, device="cuda")
        it = torch.empty(J, dtype=torch.int32, device="cuda")
        h.eval_likelihood_device(0, J, theta.data_ptr(), G.data_ptr(), Phi.data_ptr(), it.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert int(it.min()) > 0, B
        out[B] = (G.cpu().numpy(), it.cpu().numpy())
    h.set_block_size(0, 0)
    assert np.abs(out[1024][1] - out[-1024][1]).max() <= 1
    assert _rel(out[-1024][0], out[1024][0]).max() < 1e-7


@pytest.mark.parametrize("inv_h,T", [(64, 512), (32, 256)])
def test_compact_form_equals_shared_memory_form(inv_h, T):
    """The compact form (several blocks per SM: five fine-level arrays, four per coarse level,
    refinement state in device memory) does the same arithmetic as the form with the whole state
    in shared memory: with the same threads per particle the potentials and iteration counts are
    bit-identical, at the benchmark's launch size."""
    import torch
    w = wl.WORKLOADS["mls2mc_mixed_h8_64"]
    d = _data(w.name)
    h = native.Handle([inv_h], w.K, wl.obs_grid(7), d["y"], d["sigma"], corr_len=w.corr_len,
                      precision=native.SMC_MIXED)
    theta = torch.from_numpy(wl.particles(w.J, w.K, 808)).cuda()
    out = {}
    for B in (T, -T):
        h.set_block_size(0, B)
        Phi = torch.empty(w.J, dtype=torch.float64, device="cuda")
        it = torch.empty(w.J, dtype=torch.int32, device="cuda")
        h.eval_likelihood_device(0, w.J, theta.data_ptr(), 0, Phi.data_ptr(), it.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert int(it.min()) > 0
        out[B] = (Phi.cpu().numpy(), it.cpu().numpy())
    h.set_block_size(0, 0)
    assert np.array_equal(out[T][0], out[-T][0]) and np.array_equal(out[T][1], out[-T][1])


@pytest.mark.parametrize("prec", [native.SMC_MIXED, native.SMC_FP64])
def test_maximum_terms_and_observations(prec):
    """The largest problem the descriptor admits per particle: K = 256 KL terms and 1024
    observations (a 32 x 32 interpolated grid) on 1/h = 16, against the oracle."""
    K, N = 256, 16
    obs = wl.obs_grid(32)
    assert obs.shape[0] == 1024
    theta = wl.particles(3, K, 404) * 0.3
    y = np.zeros(1024)
    h = native.Handle([N], K, obs, y, 1.0, corr_len=0.1, precision=prec)
    G, _ = h.eval_likelihood(0, theta)
    lv = ofwd.Level(N, 0.1, 1.0, K, obs)
    Gr = lv.G_batch(theta)
    tol = 1e-6 if prec == native.SMC_MIXED else 1e-10
    assert _rel(G, Gr).max() < tol
