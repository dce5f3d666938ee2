"""The C ABI: the library loads, exports every function include/mls2mc.h declares,
and rejects invalid descriptors before touching the GPU (no compute calls here)."""
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
           dict(inv_h=[16], K=65, cov="matern"),                       # Matern KL keeps <= 64 terms
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
