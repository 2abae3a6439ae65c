"""gbfmm: a GB300-native (sm_103a) fast multipole method for 3-D Laplace.

The compute path is the C-ABI library ``libgbfmm.so`` built from ``csrc/``
(hand-written CUDA kernels); :mod:`.fmm` is a thin ctypes binding over it and
:mod:`.workloads` holds the seeded input generators.  Importing this package
loads nothing; the library is loaded on first use and a missing library is
an error, never a fallback.
"""

__all__ = ["workloads"]
