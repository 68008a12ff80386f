"""GB300-native Monte Carlo of the 3D Edwards-Anderson Heisenberg spin glass
(checkerboard heat-bath / over-relaxation sweeps and parallel tempering,
Yavors'kii & Weigel, arXiv:1204.6192).

The compute path is the CUDA library ``libhsg.so`` behind ``include/hsg.h``;
``hsg`` is its ctypes binding and ``inputs`` draws seeded disorder.  Importing
the package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
from .hsg import Context, HsgError, PRECISIONS, lib  # noqa: F401

__all__ = ["Context", "HsgError", "PRECISIONS", "lib"]
