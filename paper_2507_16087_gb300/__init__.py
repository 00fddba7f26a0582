"""GB300-native split-preconditioned Born solver for the heterogeneous-density
acoustic Helmholtz equation (first-order velocity/pressure system).

The compute path lives in the CUDA library under ``csrc/`` (C ABI declared in
``include/cbs.h``); ``cbs`` is the thin ctypes binding.  ``workloads`` builds
seeded synthetic inputs.  Importing this package loads nothing; the CUDA
library is loaded (and must be present) on first use of ``cbs``.
"""
__all__ = ["cbs", "workloads"]
