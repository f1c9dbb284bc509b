"""GB300-native matrix repartitioning: LDU merge, in-place value update and
Jacobi-PCG on one device CSR matrix (arXiv 2510.08536, Sec. 3-4).

Submodules:
  repart  -- binding of the C ABI (librepart.so, hand-written CUDA)
  build   -- nvcc build of librepart.so for sm_103a
  synth   -- seeded synthetic meshes, decompositions and coefficients
"""
