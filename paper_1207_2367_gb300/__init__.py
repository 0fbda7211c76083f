"""GB300 (sm_103a) engine for the direct-summation, 6th-order Hermite block-timestep
N-body method of Capuzzo-Dolcetta, Spera & Punzo (HiGPUs).

The C ABI lives in include/hg.h and the CUDA library in csrc/; `binding`
exposes the same calls to Python.  `inputs` draws the seeded synthetic
initial conditions.  Importing the package loads nothing: the CUDA library is
built and loaded on the first `binding.load()`.
"""
