"""The batched sampler: many problems' MLS^2MC (and single-level SMC) runs advanced together, every
problem's next importance-sampling update in shared launches (Sec. 4.4 update scheme, Sec. 3.4
increments, Sec. 2.4 resampling). Each problem's path, evidence and particles must equal those of
its own handle stepped alone, bit for bit (the same kernels per problem), on the FP64 and on the
mixed path, with problems of different hierarchies, K, J, seeds, kernels and schemes in one batch."""
import numpy as np
import pytest
import torch

from oracle import forward as ofwd
from paper_1709_09763_gb300 import native
from paper_1709_09763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1709_09763_gb300 import build
    build.build()


def _data(levels, K, lc, seed):
    """y = G of a prior draw on a mesh twice as fine as the finest level (oracle), 2 % noise."""
    obs = wl.obs_grid(7)
    lv = ofwd.Level(2 * levels[-1], lc, 1.0, K, obs)
    g = lv.G(wl.standard_normals((K,), seed))
    sigma = 0.02 * float(np.abs(g).max())
    return obs, g + sigma * wl.standard_normals((49,), seed + 1), sigma


def _specs(prec):
    if prec == native.SMC_FP64:
        return [dict(levels=(4, 8, 16), K=8, lc=0.3, J=300, seed=11),
                dict(levels=(8,), K=4, lc=0.3, J=200, seed=12),
                dict(levels=(4, 8, 16, 32), K=12, lc=0.2, J=257, seed=13, proposal="rwm", s_pcn=0.5),
                dict(levels=(8, 16), K=6, lc=0.3, J=150, seed=14, tau_min=0.3),
                dict(levels=(4, 8), K=5, lc=0.3, J=180, seed=15, accept_target=0.3)]
    return [dict(levels=(8, 16, 32), K=16, lc=0.2, J=400, seed=21),
            dict(levels=(16, 32, 64), K=32, lc=0.1, J=333, seed=22),
            dict(levels=(32,), K=8, lc=0.3, J=128, seed=23),
            dict(levels=(8, 16, 32, 64), K=24, lc=0.1, J=512, seed=24, accept_target=0.25)]


def _kwargs(sp, prec, stream):
    obs, y, sigma = _data(sp["levels"], sp["K"], sp["lc"], 100 + sp["seed"])
    return dict(inv_h=list(sp["levels"]), K=sp["K"], obs_xy=obs, y=y, sigma=sigma, corr_len=sp["lc"], J=sp["J"],
                J_tilde=64, n_mcmc=3, precision=prec, seed=sp["seed"], stream=stream,
                proposal=sp.get("proposal", "pcn"), s_pcn=sp.get("s_pcn", 0.2), tau_min=sp.get("tau_min", 0.0),
                accept_target=sp.get("accept_target", 0.0))


def _handle(kw):
    kw = dict(kw)
    return native.Handle(kw.pop("inv_h"), kw.pop("K"), kw.pop("obs_xy"), kw.pop("y"), kw.pop("sigma"), **kw)


def _same_run(hb, hs):
    pb, ps = hb.path(), hs.path()
    assert len(pb) == len(ps)
    for a, c in zip(pb, ps):
        for k in ("type", "level", "beta", "zeta", "delta", "cv", "cv_lu", "log_z_inc", "accept_rate",
                  "evals_per_level", "n_bridge", "n_unique", "step"):
            assert a[k] == c[k], (k, a[k], c[k])
    tb, fb = hb.particles()
    ts, fs = hs.particles()
    assert np.array_equal(tb, ts) and np.array_equal(fb, fs)
    assert hb.state() == hs.state()
    assert hb.posterior_moments()[2] == hs.posterior_moments()[2]


@pytest.mark.parametrize("prec", [native.SMC_FP64, native.SMC_MIXED])
def test_batched_runs_equal_single_handle_runs(prec):
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    kws = [_kwargs(sp, prec, s) for sp in _specs(prec)]
    batch_handles = [_handle(kw) for kw in kws]
    b = native.Batch(batch_handles)
    steps = 0
    while True:
        infos = b.step()
        steps += 1
        if all(i["status"] == 1 for i in infos):
            break
        assert steps < 500
    singles = [_handle(kw) for kw in kws]
    for h in singles:
        h.run()
    for hb, hs in zip(batch_handles, singles):
        _same_run(hb, hs)
        assert hs.state()["n_updates"] > 0
    # the multilevel problems went through level updates (bridging) and finished on their top level
    assert any(p["type"] == 1 for p in batch_handles[0].path())
    b.close()
    for h in batch_handles + singles:
        h.close()


def test_init_batch_owns_its_handles_and_runs_to_the_posterior():
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    kws = [_kwargs(sp, native.SMC_MIXED, s) for sp in _specs(native.SMC_MIXED)[:2]]
    b = native.init_batch(kws)
    n = b.run()
    assert n > 0
    for hb, kw in zip(b.handles, kws):
        hs = _handle(kw)
        hs.run()
        _same_run(hb, hs)
        st = hb.state()
        assert st["beta"] == 1.0 and st["level"] == len(kw["inv_h"]) - 1
        hs.close()
    # a further run has nothing to do
    assert b.run() == 0
    b.close()


def test_batched_sampler_rejects_what_it_does_not_run():
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    sp = _specs(native.SMC_MIXED)[2]
    h1 = _handle(_kwargs(sp, native.SMC_MIXED, s1.cuda_stream))
    h2 = _handle(_kwargs(dict(sp, seed=31), native.SMC_MIXED, s2.cuda_stream))
    b = native.Batch([h1, h2])
    with pytest.raises(native.SmcError) as e:
        b.step()
    assert e.value.code == native.SMC_EINVAL
    b.close()
    kw = _kwargs(sp, native.SMC_MIXED, s1.cuda_stream)
    kw["surrogate"] = 2
    h3 = _handle(kw)
    kw = _kwargs(sp, native.SMC_MIXED, s1.cuda_stream)
    kw["proposal"] = "rwm_cov"
    h4 = _handle(kw)
    for h in (h3, h4):   # the screened sampler and the covariance-shaped walk run per handle only
        b = native.Batch([h])
        with pytest.raises(native.SmcError) as e:
            b.step()
        assert e.value.code == native.SMC_EINVAL
        b.close()
    for h in (h1, h2, h3, h4):
        h.close()
