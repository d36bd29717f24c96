"""GB300 (sm_103a) TL-FEA hot path: internal force, tangent product, adjoint
and batched Newton/CG step of the Total Lagrangian formulation, as CUDA
kernels behind the C ABI of include/tlfe.h.

Importing this package does not load the CUDA library; `tlfe.load()` (called
by every operation) does, and raises if it has not been built.
"""

from . import tlfe  # noqa: F401
from .tlfe import Mesh, TLFEError, T4, T10, H8, SVK, NEOHOOKE, FP32, FP64, SCATTER_ATOMIC, SCATTER_COLOR  # noqa: F401
