"""GB300 (sm_103a) library for the Newton-Krylov / Chebyshev-Arnoldi stability analysis of air
convection in a laterally heated cube.  The compute path is libcubefv.so (C-ABI in
include/cube_fv.h); `fv` is its ctypes binding, `seeded` the shared synthetic-input generator.
Submodules are imported explicitly, so importing the package loads no CUDA code."""
