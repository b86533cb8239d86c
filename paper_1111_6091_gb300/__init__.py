"""GB300-native multigrid CP-ALS (De Sterck & Miller's adaptive algebraic multigrid for
low-rank canonical tensor decomposition).

* ``cpmg``  — ctypes binding of libcpmg (include/cpmg.h); the CUDA library is loaded
  on first use and its absence is an error.
* ``synth`` — seeded synthetic inputs (collinear-factor tensors, initial guesses).
* ``build`` — in-tree nvcc build of libcpmg.so for sm_103a.
"""
__all__ = ["cpmg", "synth", "build"]
