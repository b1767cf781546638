"""GB300 (sm_103a) implementation of the Immersed Boundary Double Layer
method's GMRES hot path (Leathers & Guy, arXiv:2203.12126).

The computation lives in the CUDA library ``libibdl.so`` behind the C ABI of
``include/ibdl.h``; ``ibdl`` is its ctypes binding.  There is no CPU
fallback: loading fails loudly if the library has not been built.
"""
from . import ibdl  # noqa: F401
from .ibdl import (DIRICHLET, FP32_REFINED, FP64, NEUMANN, Geometry,  # noqa: F401
                   IbdlError, Server, kernel_launch_count, load)
