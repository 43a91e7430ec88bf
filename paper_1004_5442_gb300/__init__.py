"""GB300 (sm_103a) library for the D2V16 thermal MRT finite-difference lattice
Boltzmann step of Chen, Xu, Zhang, Li and Succi (arXiv:1004.5442).

Submodules:
  build     - compiles csrc/*.cu into _build/libmrtfdlb.so (nvcc, sm_103a)
  binding   - ctypes binding of the C ABI (include/mrtfdlb.h)
  workloads - seeded synthetic initial states shaped like the paper's problems

Importing the package loads nothing; ``binding.load()`` loads the CUDA
library and raises if it has not been built.
"""
