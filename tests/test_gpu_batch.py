"""Many independent problems in one persistent launch per level size (1/128 in the two-CTA form,
1/256 in the device-memory form: the forms single solves default to), captured in a CUDA graph:
every problem's potentials equal its own single-problem evaluation bit for bit (same per-particle
solve), in eager mode, on the first graph launch and on replays with new particle values."""
import numpy as np
import pytest
import torch

from paper_1709_09763_gb300 import native
from paper_1709_09763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _problems():
    rng = np.random.default_rng(7)
    specs = [((8, 16, 32), 16, 0.3, native.SMC_MIXED), ((16, 32, 64), 32, 0.1, native.SMC_MIXED),
             ((8, 16), 8, 0.3, native.SMC_FP64), ((16, 64), 64, 0.1, native.SMC_MIXED),
             ((32,), 16, 0.3, native.SMC_MIXED), ((8, 32), 32, 0.1, native.SMC_FP64),
             ((16, 128), 16, 0.3, native.SMC_MIXED), ((32, 128), 32, 0.1, native.SMC_MIXED),
             ((256,), 32, 0.1, native.SMC_MIXED)]
    hs = []
    for levels, K, lc, prec in specs:
        obs = wl.obs_grid(7)
        y = rng.normal(0.02, 0.005, 49)
        hs.append(native.Handle(list(levels), K, obs, y, 0.002, corr_len=lc, precision=prec))
    return hs, rng


def test_batch_matches_single_problem_evaluations():
    hs, rng = _problems()
    stream = torch.cuda.Stream()
    levels = [2, 1, 1, 1, 0, 1, 1, 1, 0]
    counts = [37, 400, 129, 250, 1, 77, 9, 300, 2]
    b = native.Batch(hs)
    with torch.cuda.stream(stream):
        th = [torch.from_numpy(rng.normal(0, 1, (n, h.K))).cuda() for h, n in zip(hs, counts)]
        ph = [torch.empty(n, dtype=torch.float64, device="cuda") for n in counts]
        it = [torch.empty(n, dtype=torch.int32, device="cuda") for n in counts]

    def single():
        out = []
        for h, l, t in zip(hs, levels, th):
            _, phi = h.eval_likelihood(l, t.cpu().numpy(), want_G=False)
            out.append(phi)
        return out

    for use_graph in (False, True, True):
        for t in th:
            t.normal_()
        ref = single()
        b.eval(levels, counts, [t.data_ptr() for t in th], [p.data_ptr() for p in ph],
               [i.data_ptr() for i in it], stream.cuda_stream, use_graph)
        stream.synchronize()
        for p, r, i in zip(ph, ref, it):
            assert np.array_equal(p.cpu().numpy(), r)
            assert int(i.min()) > 0
    b.close()
