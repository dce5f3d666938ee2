"""GB300 (sm_103a) library for the likelihood hot path of Multilevel Sequential^2 Monte Carlo.

Latz, Papaioannou, Ullmann, arXiv:1709.09763. The compute path lives in the CUDA
library libmls2mc.so (C ABI in include/mls2mc.h); `native` is its thin ctypes
binding and `build` compiles it in-tree. `workloads` holds the synthetic
workload definitions and seeded input draws.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "native", "build"]
