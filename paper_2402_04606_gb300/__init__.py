"""GB300 (sm_103a) library for the hot path of SBoTFlow (arXiv 2402.04606):
the fused D2Q9 stream-collide sweep over a block-refined grid, the coarse/fine
interface transfers, the multi-direct-forcing immersed boundary and the
drag/lift/moment reduction.

The compute path is the C-ABI library ``libsbot.so`` (CUDA kernels in
``csrc/``); ``native`` is its ctypes binding and ``workloads`` holds the
seeded synthetic workload parameters.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "native", "build"]
