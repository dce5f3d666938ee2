"""The stored data vectors under tests/golden/ are what the committed generator writes from the
oracle alone (make_golden.py: a seeded prior draw, the oracle's FP64 forward solve on the data
mesh, seeded noise), re-derived here for the workloads whose data mesh solves in seconds."""
import json
import os
import sys

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLD)

import make_golden                                      # noqa: E402
from paper_1709_09763_gb300 import workloads as wl      # noqa: E402


@pytest.mark.parametrize("name", ["smc_fp64_h16", "mls2mc_mixed_h8_64", "example_5_1", "example_5_2",
                                  "example_5_3"])
def test_stored_data_come_from_the_oracle(name):
    with open(os.path.join(GOLD, f"data_{name}.json")) as f:
        stored = json.load(f)
    d = make_golden.make(wl.WORKLOADS[name])
    assert d["inv_h_data"] == stored["inv_h_data"]
    assert np.array_equal(d["theta_true"], stored["theta_true"])
    assert d["sigma"] == pytest.approx(stored["sigma"], rel=1e-12)
    assert np.allclose(d["G_data"], stored["G_data"], rtol=0, atol=1e-12)
    assert np.allclose(d["y"], stored["y"], rtol=0, atol=1e-12)
