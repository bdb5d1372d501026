"""GB300-native (sm_103a) FP64 implementation of the fifth-order finite-difference
interpolation-based Hermite WENO scheme HWENO-I (Xie, Tao, Jiao, Zhang, arXiv 2411.11229).

The numerical work runs in libhweno.so (CUDA, see include/hweno.h); this package only builds
and loads it and marshals torch-owned device memory into its C ABI.  HWENO_BOUNDS_CHECK=1 in the
environment selects the bounds-checked build of the same sources, libhweno_bounds.so.
"""
from ._make import build, build_all  # noqa: F401


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver
        return Solver
    if name == "Batch":
        from .solver import Batch
        return Batch
    if name == "capi":
        from . import _capi
        return _capi
    raise AttributeError(name)
