"""The allocation-free resampling entry point against the handle-based one.

smc_systematic_resample_noalloc exists for callers that cannot allocate device memory (their
device memory belongs to another framework's pool, or cudaMalloc is not allowed once they run).
Its scratch is a fixed device array shared by all calls, so two calls in a row -- the second one
smaller -- must each give exactly the indices of smc_systematic_resample, and a size beyond the
array must be rejected. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1709_09763_gb300 import native

pytestmark = pytest.mark.gpu


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
        rc = lib.smc_systematic_resample_noalloc(ctypes.c_void_p(w_dev.data_ptr()), n, U,
                                                 ctypes.c_void_p(anc_dev.data_ptr()), ctypes.c_void_p(stream))
        torch.cuda.synchronize()
        assert rc == native.SMC_OK
        assert np.array_equal(anc_dev.cpu().numpy(), ref)       # index work: bit-exact
    # more particles than the fixed scratch holds: rejected before any launch
    big = native.SMC_NOALLOC_MAX_PARTICLES + 1
    rc = lib.smc_systematic_resample_noalloc(ctypes.c_void_p(w_dev.data_ptr()), big, 0.5,
                                             ctypes.c_void_p(anc_dev.data_ptr()), ctypes.c_void_p(stream))
    assert rc == native.SMC_EINVAL
