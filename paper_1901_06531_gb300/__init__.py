"""GB300-native Galerkin FFT homogenization with stress and mixed control
(Lucarini & Segurado, arXiv:1901.06531).

Submodules:
  inputs -- seeded synthetic microstructures, orientations and load histories
  build  -- nvcc build of the CUDA library libmixfft.so (sm_103a)
  mixfft -- ctypes binding of the C ABI (include/mixfft.h); importing it
            requires the built library
"""
