"""GB300-native phase-field thermocapillary lattice Boltzmann (arXiv 2306.11320).

Submodules:
  tpflbm     ctypes binding of the CUDA C-ABI library (libtpflbm.so)
  workloads  seeded synthetic parameters and initial fields
  build      in-tree nvcc build of the CUDA library
Importing the package itself loads nothing.
"""
