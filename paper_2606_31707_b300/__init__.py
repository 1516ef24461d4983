"""B300 (sm_103a) implementation of the HLBM mean-flow adjoint hot path.

The compute path is the CUDA library ``libhlbm.so`` built from ``csrc/``
(see ``include/hlbm.h`` for the C ABI); ``hlbm`` is its ctypes binding with
the C names, ``Solver`` a per-context convenience wrapper.  Importing this
package fails if the library has not been built.
"""
from . import hlbm
from .hlbm import HlbmError
from .solver import Solver

__all__ = ["hlbm", "HlbmError", "Solver"]
