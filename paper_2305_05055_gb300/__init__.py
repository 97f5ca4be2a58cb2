"""GPU (sm_103a) CPMA: a batch-parallel compressed set of 64-bit keys.

``cpma`` is the binding of the C ABI in ``include/cpma.h``; ``workloads`` holds
the seeded synthetic input generators.
"""
from . import workloads  # noqa: F401

__all__ = ["cpma", "workloads", "build"]
