"""GB300-native Fourier split-operator propagator (Bauke & Keitel, arXiv:1012.3911).

The hot path lives in ``libsop.so`` (hand-written CUDA for sm_103a behind the
``sop_*`` C ABI declared in ``include/sop.h``).  This package holds the thin
ctypes binding (``sop``), the in-tree build step (``build``), the seeded
input generators (``workloads``) and the replica bookkeeping of multi-GPU runs
(``replicas``).  Importing the package does not load the
CUDA library; the binding loads it on first use and fails loudly if it is
missing.
"""
__all__ = ["sop", "workloads", "build", "replicas"]
