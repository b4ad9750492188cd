"""GB300 (sm_103a) implementation of the asymptotic-preserving IMEX-RK scheme
for the six-velocity lattice-Boltzmann-type DVM in the low-Mach scaling.

The compute path is the CUDA library ``libapdvm.so`` (C ABI in
``include/ap_dvm.h``); ``api`` is its ctypes binding, ``workloads`` the seeded
input generators.  Importing the package loads nothing; ``api.lib()`` loads
the library and raises if it is missing.
"""
__all__ = ["api", "workloads", "tableaux"]
