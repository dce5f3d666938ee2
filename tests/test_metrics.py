"""Accuracy measures of Sec. 5.1 (RelErr, RelMisfit, KS distance, RelErrEvid) on hand-computed
cases and against scipy's two-sample KS statistic."""
import numpy as np
import pytest

from paper_1709_09763_gb300 import metrics


def test_rel_err_hand_values():
    lam = np.array([4.0, 1.0])                    # weights 2, 1
    assert metrics.rel_err([1.0, 1.0], [1.0, 1.0], lam) == 0.0
    # |2 (0 - 1)| + |1 (3 - 1)| = 4 over 2 |1| + 1 |1| = 3
    assert metrics.rel_err([0.0, 3.0], [1.0, 1.0], lam) == pytest.approx(4.0 / 3.0)


def test_rel_misfit_from_potential():
    y, sigma = np.array([1.0, -2.0, 2.0]), 0.5
    G = np.array([0.5, -2.0, 1.0])
    phi = 0.5 * np.sum(((y - G) / sigma) ** 2)
    want = np.sum(((y - G) / sigma) ** 2) / np.sum((y / sigma) ** 2)
    assert metrics.rel_misfit(phi, y, sigma) == pytest.approx(want, rel=1e-15)


def test_ks_distance_against_scipy_and_limits():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(0)
    for n, m, shift in ((100, 100, 0.0), (250, 97, 0.3), (5, 9, 1.0)):
        a, b = rng.normal(0, 1, n), rng.normal(shift, 1, m)
        assert metrics.ks_distance(a, b) == pytest.approx(stats.ks_2samp(a, b).statistic, abs=1e-15)
    a = rng.normal(0, 1, 50)
    assert metrics.ks_distance(a, a) == 0.0
    assert metrics.ks_distance(a, a + 100.0) == 1.0
    # ties: resampled particles repeat values
    assert metrics.ks_distance([1, 1, 2, 2], [1, 2, 2, 2]) == pytest.approx(0.25)


def test_evidence_reference_and_relative_error():
    lz = np.array([-10.0, -12.0, -11.0])
    ref = metrics.log_z_ref(lz)
    assert ref == -11.0                            # log of the geometric mean of exp(lz)
    assert np.allclose(metrics.rel_err_evid(lz, ref), [1 / 11, 1 / 11, 0.0])


def test_pairwise_ks_counts_and_symmetry():
    rng = np.random.default_rng(1)
    runs = [rng.normal(0, 1, (40, 3)) for _ in range(4)]
    mean, sd, n = metrics.pairwise_ks(runs)
    assert n == 6 and mean.shape == (3,) and np.all(mean > 0) and np.all(sd >= 0)
    mean2, _, n2 = metrics.pairwise_ks(runs[:2], runs[2:])
    assert n2 == 4
    d = [metrics.ks_distance(runs[i][:, 0], runs[j][:, 0]) for i in (0, 1) for j in (2, 3)]
    assert mean2[0] == pytest.approx(np.mean(d))
