"""GB300-native flux reconstruction stochastic Galerkin (FR-SG) library.

The compute path is the CUDA library libfrsg.so (C ABI in include/frsg.h), built
in-tree for sm_103a by build.build(); frsg.Solver is a thin ctypes binding of it.
workloads holds the seeded synthetic problem definitions shared by the tests, the
benchmark and the smoke check.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "frsg", "build"]
