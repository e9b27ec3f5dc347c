"""GB300-native monolithic multigrid for fully implicit Runge-Kutta stage
systems of incompressible flow (Abu-Labdeh, MacLachlan & Farrell,
arXiv:2202.07381).

The compute path is the CUDA library `libirkmg.so` (sources in csrc/, C ABI in
include/irkmg.h); `irkmg` is a thin ctypes binding with the same names.
Importing this package loads nothing; the library is opened on first use and
raises if it has not been built.
"""
__all__ = ["irkmg", "build"]
