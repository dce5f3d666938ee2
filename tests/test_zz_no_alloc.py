"""The allocation-free resampling entry point against the handle-based one and the oracle.

smc_systematic_resample_noalloc exists for callers that cannot allocate device memory (their
device memory belongs to another framework's pool, or cudaMalloc is not allowed once they run).
Its scratch is a fixed device array shared by all calls, so two calls in a row -- the second one
smaller -- must each give exactly the indices of smc_systematic_resample, dyadic weights (every
partial sum exact in any order) must give the oracle's indices bit for bit, the device's free
memory must not change across a call, and a size beyond the array, n = 0 and an offset outside
[0, 1) must be rejected. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle import smc as osmc
from paper_1709_09763_gb300 import native

pytestmark = pytest.mark.gpu


def _call(lib, w_dev, n, U, anc_dev, stream):
    return lib.smc_systematic_resample_noalloc(ctypes.c_void_p(w_dev.data_ptr()), n, U,
                                               ctypes.c_void_p(anc_dev.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_resampling_matches_handle_entry_point_twice():
    import torch
    from paper_1709_09763_gb300 import build
    build.build()
    lib = native.load()
    n_max = 6000
    A = np.ones((1, 1, 2))
    h = native.Handle([4], 2, np.full((1, 2), 0.5), np.zeros(1), 1.0, J=n_max, linear_A=A)
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream().cuda_stream
    for n, U in ((5000, 0.3141592653589793), (1234, 0.75)):
        w = np.exp(rng.normal(0.0, 2.0, n))
        ref = h.systematic_resample(w, U)
        w_dev = torch.from_numpy(w).cuda()
        anc_dev = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = _call(lib, w_dev, n, U, anc_dev, stream)
        torch.cuda.synchronize()
        assert rc == native.SMC_OK
        assert np.array_equal(anc_dev.cpu().numpy(), ref)       # index work: bit-exact
    # more particles than the fixed scratch holds: rejected before any launch
    big = native.SMC_NOALLOC_MAX_PARTICLES + 1
    assert _call(lib, w_dev, big, 0.5, anc_dev, stream) == native.SMC_EINVAL
    # no particles, an offset outside [0, 1), NaN: rejected
    assert _call(lib, w_dev, 0, 0.5, anc_dev, stream) == native.SMC_EINVAL
    assert _call(lib, w_dev, 10, 1.0, anc_dev, stream) == native.SMC_EINVAL
    assert _call(lib, w_dev, 10, -0.25, anc_dev, stream) == native.SMC_EINVAL
    assert _call(lib, w_dev, 10, float("nan"), anc_dev, stream) == native.SMC_EINVAL
    h.close()


def test_noalloc_resampling_equals_oracle_on_dyadic_weights_and_allocates_nothing():
    import torch
    lib = native.load()
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(native.SMC_NOALLOC_MAX_PARTICLES, 0.0), (4096, 0.5), (1000, 0.123456789), (7, 0.999)]
    bufs = []
    for n, U in cases:
        w = 2.0 ** rng.integers(-12, 0, size=n)
        bufs.append((n, U, w, torch.from_numpy(w).cuda(), torch.full((n,), -1, dtype=torch.int32, device="cuda")))
    torch.cuda.synchronize()
    for i, (n, U, w, w_dev, anc_dev) in enumerate(bufs):
        free0 = torch.cuda.mem_get_info()[0]
        rc = _call(lib, w_dev, n, U, anc_dev, stream)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert rc == native.SMC_OK
        assert np.array_equal(anc_dev.cpu().numpy(), osmc.systematic_resample(np.log(w), U)), (n, U)
        if i > 0:                   # after a first call (which may load device code): no allocation
            assert free1 == free0
