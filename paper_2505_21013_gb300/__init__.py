"""GB300 (sm_103a) Progressively Projected Newton: per-Newton-iteration element
pipeline of implicit-Euler tetrahedral FEM as hand-written CUDA kernels behind a
C ABI (``include/ppn.h``).  ``ppn`` is the ctypes binding; ``build`` compiles
``libppn.so`` in-tree.
"""

from . import ppn  # noqa: F401
from .ppn import (MODE_NEWTON, MODE_PDN, MODE_PN, MODE_PPN, PCG_LAYOUTS, PREC_FP64, PREC_MIXED,  # noqa: F401
                  PROJ_CLAMP, PROJ_MIRROR, PPNError, Scene, Server, ppn_default_params, ppn_step_batch)

__all__ = ["ppn", "Scene", "Server", "PPNError", "ppn_default_params", "ppn_step_batch", "MODE_NEWTON", "MODE_PN",
           "MODE_PPN", "MODE_PDN", "PCG_LAYOUTS", "PROJ_CLAMP", "PROJ_MIRROR", "PREC_FP64", "PREC_MIXED"]
