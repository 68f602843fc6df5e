"""GB300 (sm_103a) MinxEnt-LBM: the fused stream-and-collide time step of
Wilson, Pugh & Dawson, "Stabilization of the Lattice Boltzmann Method Using
Information Theory" (arXiv:1801.03863), behind the C ABI of include/lbm.h.

Modules:
  lbm        ctypes binding of liblbm.so (same names as the C entry points)
  workloads  seeded synthetic initial fields and ensemble parameters
  _build     nvcc build of liblbm.so for sm_103a
"""
from . import workloads  # noqa: F401

__all__ = ["lbm", "workloads"]
