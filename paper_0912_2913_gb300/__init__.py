"""GB300-native relativistic lattice Boltzmann (arXiv:0912.2913): the fused
stream-and-collide step, its macroscopic output and its discrete adjoint, as
hand-written sm_103a CUDA behind the C ABI of include/rlb.h."""
from . import _native
from ._native import RLBError
from .autograd import RunSpec, rlb_run
from .rlb import RLB

__all__ = ["RLB", "RLBError", "RunSpec", "rlb_run", "_native"]
