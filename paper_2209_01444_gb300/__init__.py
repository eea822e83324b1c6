"""GB300-native (sm_103a) diffuse-interface MRT lattice Boltzmann method for
dendritic growth with thermosolutal convection (arXiv 2209.01444).

Modules:
  lbm        ctypes binding of the C ABI (include/lbm.h) and a Simulation class;
  workloads  seeded synthetic problem statements (parameters, seeds, fields);
  build_ext  nvcc build of liblbm.so.
Importing the package loads nothing; ``lbm.load()`` loads the CUDA library.
"""
