"""The C ABI: the library loads, exports every function include/mls2mc.h declares,
rejects invalid descriptors before touching the GPU, and builds the KL tables of its host
set-up (Eq. truncKL; the Matern prior of Sec. 5) equal to the oracle's. No GPU call here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1709_09763_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(smc_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1709_09763_gb300 import build
    build.build()
    return native.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "smc_eval_likelihood" in names and "smc_init" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(native.SIGNATURES) >= names


def test_invalid_descriptors_rejected_without_gpu(lib):
    obs = np.array([[0.5, 0.5]])
    y = np.zeros(1)
    bad = [dict(inv_h=[16], K=0), dict(inv_h=[16], K=300), dict(inv_h=[12], K=4),
           dict(inv_h=[16, 8], K=4), dict(inv_h=[16], K=4, sigma=0.0),
           dict(inv_h=[16], K=4, obs_xy=np.array([[1.5, 0.5]])),
           dict(inv_h=[16], K=513, cov="matern", precision=native.SMC_MIXED),  # Matern KL: <= 512 terms
           dict(inv_h=[16], K=513, precision=native.SMC_MIXED),        # mixed FEM path: K <= 512
           dict(inv_h=[16, 64], K=4, bc="flow_cell", precision=native.SMC_FP64),   # FP64 flow cell to 1/32
           dict(inv_h=[16], K=4, bc="flow_cell", source="nine")]       # flow cell: f = 0
    for kw in bad:
        args = dict(obs_xy=obs, y=y, sigma=1.0)
        args.update(kw)
        with pytest.raises(native.SmcError) as ei:
            native.Handle(**args)
        assert ei.value.code == native.SMC_EINVAL, kw
    # FP64 path stops at 1/h = 32 (on-chip FP64 hierarchy)
    with pytest.raises(native.SmcError) as ei:
        native.Handle(inv_h=[64], K=4, obs_xy=obs, y=y, sigma=1.0, precision=native.SMC_FP64)
    assert ei.value.code == native.SMC_EINVAL


@pytest.mark.parametrize("N,lc,K", [(8, 0.65, 10), (32, 0.65, 10), (16, 0.1, 64), (16, 0.1, 65), (16, 0.1, 320)])
def test_host_matern_table_equals_oracle(lib, N, lc, K):
    """The library's Nystrom KL (its own eigen-solver and symmetry reduction) against the oracle's
    (LAPACK on the same sub-problems): every table entry and eigenvalue, up to rounding."""
    from oracle import matern
    psi, lam = native.kl_table_host("matern", N, lc, 1.0, K)
    assert np.abs(psi - matern.kl_table(N, lc, 1.0, K)).max() < 1e-12
    assert np.allclose(lam, matern.eigenvalues(lc, 1.0, K), rtol=0, atol=1e-15)


def test_host_matern_table_320_terms_on_a_fine_level(lib):
    """Example 5.3's 320 terms on 1/128, sampled elements (the oracle extends them one by one)."""
    from oracle import matern
    N = 128
    psi, lam = native.kl_table_host("matern", N, 0.1, 1.0, 320)
    el = np.random.default_rng(3).choice(2 * N * N, 200, replace=False)
    assert np.abs(psi[:, el] - matern.kl_table_at(N, el, 0.1, 1.0, 320)).max() < 1e-12
    assert 0.945 < lam.sum() < 0.955


def test_host_sep_exp_table_and_invalid_arguments(lib):
    from oracle import kl
    psi, lam = native.kl_table_host("sep_exp", 16, 0.3, 1.0, 16)
    assert np.abs(psi - kl.kl_table(16, 0.3, 1.0, 16)).max() < 1e-13
    for args in (("matern", 16, 0.1, 1.0, 513), ("matern", 0, 0.1, 1.0, 4), ("matern", 16, 0.0, 1.0, 4),
                 ("sep_exp", 16, 0.3, -1.0, 4), ("matern", 512, 0.1, 1.0, 4), ("sep_exp", 8, 0.3, 1.0, 513)):
        with pytest.raises(native.SmcError) as ei:
            native.kl_table_host(*args)
        assert ei.value.code == native.SMC_EINVAL, args
