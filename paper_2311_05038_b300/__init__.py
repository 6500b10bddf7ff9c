"""B300-native acoustic finite-difference propagator.

The compute path is libfd.so: hand-written sm_103a CUDA kernels behind the C
ABI of include/fd.h.  ``paper_2311_05038_b300.fd`` is its Python binding
(importing it fails if the library is not built); ``build()`` compiles it.
"""
from .build import build  # noqa: F401
