"""GB300-native implicit P-multigrid FR/CPR solver (arXiv 1908.03972).

The numerical path runs in ``lib/libpmgfr.so`` (hand-written sm_103a CUDA
kernels behind a C interface, ``include/pmgfr.h``); ``pmgfr`` is its Python
binding and ``workloads`` the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "pmgfr", "build"]
