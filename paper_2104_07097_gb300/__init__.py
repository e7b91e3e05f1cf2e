"""GB300-native Matrix Hit-and-Run (arXiv 2104.07097): z walkers sampling
{x : A x <= b, A_E x = b_E} with hand-written sm_103a CUDA kernels behind the
C ABI in include/mhar.h.

``mhar``      -- ctypes binding (names mirror the C ABI) and ``Sampler``;
``build``     -- nvcc build of libmhar.so (in-tree, sm_103a);
``workloads`` -- seeded synthetic polytopes shared by tests and benchmark.
"""
from . import build, workloads  # noqa: F401

__all__ = ["build", "workloads", "mhar"]
