"""GB300-native IGA collocation + fast-diagonalization preconditioned GMRES.

The computation lives in ``libiga_fd.so`` (CUDA for sm_103a, C ABI in
include/iga_fd.h); this package is its Python binding.
"""

from ._lib import IgaError, load  # noqa: F401


def __getattr__(name):
    # lazy: importing the package does not require torch or the built library
    if name in ("Problem", "GEOM", "PREC", "FACTOR"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
