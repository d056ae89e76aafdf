"""GB300-native noisy mean-field annealing (NMFA, Algorithm 1 of arXiv 1806.08422).

Submodules:
  nmfa       -- ctypes binding of libnmfa.so (include/nmfa.h), same names as the C ABI
  instances  -- seeded synthetic instances and annealing schedules (input data only)
  build      -- nvcc build of libnmfa.so for sm_103a
Importing the package loads nothing; the binding loads the library on first use.
"""
