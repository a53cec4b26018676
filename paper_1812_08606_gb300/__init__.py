"""GB300-native GMG-preconditioned FGMRES solver for the Poisson-type equation
-div(a grad phi) = f of a semi-implicit streamer-discharge scheme.

The compute path is libgmg.so (hand-written CUDA for sm_103a, C ABI in
include/gmg.h); ``gmg`` is its ctypes binding and ``autograd`` a
torch.autograd wrapper with a hand-written adjoint.
"""
from . import gmg  # noqa: F401
from .autograd import PoissonSolver  # noqa: F401

__all__ = ["gmg", "PoissonSolver"]
