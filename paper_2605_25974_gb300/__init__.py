"""GB300-native Pauli-sum outer product and canonicalisation (PauLIB, arXiv 2605.25974).

The compute path is a C-ABI shared library (``csrc/``, declared in
``include/paulib.h``) of hand-written sm_103a CUDA kernels.  ``paulib`` is
the thin ctypes binding over it; ``workloads`` holds the seeded synthetic
input generators.  Importing this package loads nothing: the library is
opened on first use of :mod:`paper_2605_25974_gb300.paulib`.
"""
__all__ = ["paulib", "workloads"]
