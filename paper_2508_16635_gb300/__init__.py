"""GB300 (sm_103a) implementation of the implicit-Coriolis rotating-shell step,
its Jacobian action and the Newton-GMRES rotating-wave solver.

The compute path is the CUDA library librsc.so (C ABI in include/rsc.h);
`rsc` is its ctypes binding.  There is no CPU fallback.
"""
from .rsc import Batch, RotatingShell, RscError, load_library, EXPORTS  # noqa: F401
