"""GB300 (sm_103a) H-matrix Gaussian log-likelihood (arXiv:1709.08625).

``hlc`` is the ctypes binding of the C ABI in ``include/hlc.h``;
``inputs`` holds the seeded synthetic workloads; ``build`` compiles the
CUDA library in-tree.  The binding is imported on demand so that the input
generators stay usable on machines without the built library.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "hlc", "build"]
